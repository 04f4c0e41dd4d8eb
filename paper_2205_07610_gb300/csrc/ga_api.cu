// ga_api.cu -- the C ABI (include/gotoh_align.h): argument checks, workspace,
// planning (encode, classify, length sort) and kernel dispatch.
#include <algorithm>
#include <memory>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/gotoh_band.h"
#include "../../include/gotoh_plan.h"
#include "ga_band.cuh"
#include "ga_banded.cuh"
#include "ga_pool.h"
#include "ga_prot.cuh"
#include "ga_serve_host.h"
#include "ga_launch.h"
#include "ga_prep.cuh"

namespace ga {

// Inter-sequence bins (columns per group = 16 * K).
static BinTable make_bins() {
  BinTable b{};
  b.n16 = kKaNumBins;
  b.n32 = kKaNumBins;
  for (int i = 0; i < kKaNumBins; ++i) {
    b.w16[i] = kKaG * kKaK[i];
    b.w32[i] = kKaG * kKaK[i];
  }
  return b;
}

// The library's own stream-ordered memory pool per device.  Its release
// threshold keeps freed workspace mapped between calls, so a call does not
// pay for mapping and unmapping hundreds of MB at every synchronisation (the
// device's default pool returns memory to the driver at each sync).  The
// pool is created on first use per device and lives until the process ends.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}

// Side streams per device for the DP launches of one call: the bins of a
// batch run as concurrent persistent kernels (forked from and joined back to
// the caller's stream with events), so that one bin's last tasks overlap the
// next bin's first.  Created on first use, kept until the process ends.
constexpr int kSideStreams = 4;
static std::mutex g_side_mu;
static cudaStream_t g_side[64][kSideStreams] = {};

cudaStream_t *side_streams_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_side_mu);
  if (!g_side[dev][0]) {
    cudaStream_t st[kSideStreams] = {};
    for (int i = 0; i < kSideStreams; ++i)
      if (cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking) != cudaSuccess) {
        for (int k = 0; k < i; ++k) cudaStreamDestroy(st[k]);
        return nullptr;
      }
    for (int i = 0; i < kSideStreams; ++i) g_side[dev][i] = st[i];
  }
  return g_side[dev];
}

cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = pool_for_current_device();
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

namespace {

struct Scoring {
  int A = 0, alpha = 0, beta = 0, smax = 0, smin = 0;
  int8_t mat[32 * 32] = {};
  uint32_t tables[16] = {};
};

// Long pairs of alphabets of <= 4 symbols run on the packed kernel when its
// relative int16 cells are exact for the scoring (sigma_max + alpha <=
// kKwMaxStep); every other long pair on the int32 kernel.
bool long_packed(const Scoring &sc, bool dna) {
  return dna && std::max(sc.smax, 0) + sc.alpha <= kKwMaxStep;
}

int check_scoring(const ga_scoring *sc, Scoring *out) {
  if (!sc) return GA_ERR_ARG;
  if (sc->alphabet_size < 1 || sc->alphabet_size > 31 || !sc->matrix) return GA_ERR_ALPHABET;
  if (sc->gap_open <= 0 || sc->gap_extend <= 0 || sc->gap_extend > sc->gap_open || sc->gap_open > 4096)
    return GA_ERR_ARG;
  const int A = sc->alphabet_size;
  out->A = A;
  out->alpha = sc->gap_open;
  out->beta = sc->gap_extend;
  out->smax = -1000;
  out->smin = 1000;
  for (int i = 0; i < A * A; ++i) {
    const int v = sc->matrix[i];
    if (v < -127) return GA_ERR_ALPHABET;
    out->mat[i] = (int8_t)v;
    out->smax = std::max(out->smax, v);
    out->smin = std::min(out->smin, v);
  }
  // Table words for alphabets of <= 4 symbols: byte c of word x is
  // sigma(x, c) (rows = query) or sigma(c, x) (rows = target); code 4 = pad.
  if (A <= 4) {
    for (int x = 0; x < A; ++x) {
      uint32_t wn = 0, ws = 0;
      for (int c = 0; c < A; ++c) {
        wn |= (uint32_t)(uint8_t)out->mat[x * A + c] << (8 * c);
        ws |= (uint32_t)(uint8_t)out->mat[c * A + x] << (8 * c);
      }
      out->tables[x] = wn;
      out->tables[8 + x] = ws;
    }
  }
  return GA_OK;
}

// Device allocations of one call, released stream-ordered.
struct Alloc {
  cudaStream_t s;
  cudaMemPool_t pool;
  std::vector<void *> ptrs;
  bool failed = false;
  explicit Alloc(cudaStream_t st) : s(st), pool(pool_for_current_device()) {}
  template <class T>
  T *get(size_t n) {
    void *p = nullptr;
    const size_t bytes = n * sizeof(T) + 256;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s)
                               : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return (T *)p;
  }
  ~Alloc() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
  }
};

// Small pinned staging area for scalar readbacks (one per host thread).
struct Pinned {
  void *p = nullptr;
  Pinned() { cudaMallocHost(&p, 4096); }
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
void *pinned_scratch() {
  thread_local Pinned pin;
  return pin.p;
}

// Device-side scalars of one call.
struct Small {
  int32_t status;
  int32_t rmax_long;
  unsigned long long cells;
  int32_t rerun_total;
  int32_t pad0;
  int32_t ranges[2 * kClassesSorted * kBins];
  int32_t counters[64];
  int32_t rerun_range[2];
  int32_t scan_partials[kScanTiles];
  int32_t invalid_q, invalid_t;
  unsigned long long band_retries, band_cells;
  int32_t max_rows;
  int32_t max_band_span;  // max over band pairs of max(m + 1, 128) x super-stages + m, saturated
};

struct Readback {
  int32_t status;
  int32_t rmax_long;
  unsigned long long cells;
  int32_t rerun_total;
  int32_t pad0;
  int32_t ranges[2 * kClassesSorted * kBins];
};

__global__ void fill_off_kernel(int64_t *off, int64_t a, int64_t b) {
  off[0] = a;
  off[1] = b;
}

__global__ void count_reruns_kernel(const int32_t *rerun_range, int32_t *total) {
  *total += rerun_range[1];
}

// Plan runs: the rerun list [0, count) as a kernel range, counted in total.
__global__ void rerun_setup_kernel(int32_t *rerun_range, int32_t *total) {
  rerun_range[0] = 0;
  *total += rerun_range[1];
}

struct Call {
  cudaStream_t s;
  Scoring sc;
  int mode;
  int nsm = 0;
  int dna = 0;
  Alloc al;
  Small *small = nullptr;
  int32_t *hist = nullptr, *cursor = nullptr;
  int64_t pairs = 0, pairs16 = 0, pairs32 = 0;
  // Launch accounting and per-DP-launch device timing (stats requested).
  bool timing = false;
  int launches = 0, dp_launches = 0;
  std::vector<cudaEvent_t> dp_ev;
  explicit Call(cudaStream_t st) : s(st), al(st) {}
  ~Call() {
    for (cudaEvent_t e : dp_ev) cudaEventDestroy(e);
  }
  void dp_begin() {
    ++launches;
    ++dp_launches;
    if (!timing) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) == cudaSuccess) {
      dp_ev.push_back(e);
      cudaEventRecord(e, s);
    }
  }
  void dp_end() {
    if (!timing) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) == cudaSuccess) {
      dp_ev.push_back(e);
      cudaEventRecord(e, s);
    }
  }
  // Concurrent DP launches: one timed region around the fork / join.
  void count_dp() {
    ++launches;
    ++dp_launches;
  }
  void dp_mark() {
    if (!timing) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) == cudaSuccess) {
      dp_ev.push_back(e);
      cudaEventRecord(e, s);
    }
  }
  float dp_ms() const {
    float tot = 0.f;
    for (size_t i = 0; i + 1 < dp_ev.size(); i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, dp_ev[i], dp_ev[i + 1]) == cudaSuccess) tot += ms;
    }
    return tot;
  }
};

int setup(Call &c) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GA_ERR_CUDA;
  if (cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GA_ERR_CUDA;
  c.dna = c.sc.A <= 4;
  c.small = c.al.get<Small>(1);
  c.hist = c.al.get<int32_t>(kNumKeys);
  c.cursor = c.al.get<int32_t>(kNumKeys);
  if (c.al.failed) return GA_ERR_OOM;
  if (cudaMemsetAsync(c.small, 0, sizeof(Small), c.s) != cudaSuccess) return GA_ERR_CUDA;
  return GA_OK;
}

// Validate + pack one sequence set.  Reads back the total residue count.
// Residue range [off[0], off[nseq]) of a set, when the caller knows it on
// the host (otherwise it is read back from the device offsets).
struct KnownRange {
  bool known = false;
  int64_t start = 0, total = 0;
};

int prepare_set(Call &c, const uint8_t *codes, const int64_t *off, int64_t nseq, uint32_t **packed,
                uint8_t **bad, int32_t *invalid, KnownRange kr = KnownRange(), uint32_t **packed5 = nullptr) {
  *bad = c.al.get<uint8_t>((size_t)nseq + 1);
  *packed = nullptr;
  if (packed5) *packed5 = nullptr;
  if (c.al.failed) return GA_ERR_OOM;
  if (nseq == 0) return GA_OK;
  // the set's residues are codes[off[0] .. off[nseq]) (off[0] > 0 when the
  // set is a chunk of a larger buffer); packed words keep absolute positions
  int64_t h0 = kr.start, h1 = kr.total;
  if (!kr.known) {
    int64_t *h = (int64_t *)pinned_scratch();
    if (cudaMemcpyAsync(h, off, sizeof(int64_t), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaMemcpyAsync(h + 1, off + nseq, sizeof(int64_t), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaStreamSynchronize(c.s) != cudaSuccess)
      return GA_ERR_CUDA;
    h0 = h[0];
    h1 = h[1];
  }
  const int64_t total = std::max<int64_t>(h1, 0);
  const int64_t start = std::min(std::max<int64_t>(h0, 0), total);
  if (c.dna) {
    *packed = c.al.get<uint32_t>((size_t)(total / 16 + 2));
    if (c.al.failed) return GA_ERR_OOM;
  }
  const int64_t nwords = (total + 15) / 16 - start / 16;
  const int64_t pblocks = std::min<int64_t>((nwords + 255) / 256, (int64_t)c.nsm * 16);
  if (packed5 && !c.dna && total > start) {
    // 5-bit words (the packing also validates the codes)
    *packed5 = c.al.get<uint32_t>((size_t)((total + 5) / 6 + 16));
    if (c.al.failed) return GA_ERR_OOM;
    const int64_t chunks = ((total + 5) / 6 - start / 6 / 8 * 8 + 7) / 8;
    const int64_t b5 = std::min<int64_t>((chunks + 255) / 256, (int64_t)c.nsm * 16);
    flat_pack5_kernel<<<(unsigned)std::max<int64_t>(b5, 1), 256, 0, c.s>>>(codes, start, total, c.sc.A,
                                                                           *packed5, invalid);
    ++c.launches;
  } else if (nwords > 0) {
    flat_pack_kernel<<<(unsigned)std::max<int64_t>(pblocks, 1), 256, 0, c.s>>>(codes, start, total,
                                                                               c.sc.A, *packed, invalid);
    ++c.launches;
  }
  validate_kernel<<<(unsigned)((nseq + 255) / 256), 256, 0, c.s>>>(codes, off, nseq, start, total,
                                                                   c.sc.A, invalid, *bad);
  ++c.launches;
  if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;
  return GA_OK;
}

struct SetView {
  const uint8_t *codes;
  const int64_t *off;
  uint32_t *packed;
  uint8_t *bad;
};

// The DP launches of one call on the device's side streams (two or more
// launches), or in order on the caller's stream.
struct DpFork {
  Call &c;
  bool on = false;
  int n = 0;
  cudaStream_t *side = nullptr;
  cudaEvent_t fork = nullptr, join[kSideStreams] = {};
  explicit DpFork(Call &cc) : c(cc) {}
  int begin(int nlaunch) {
    if (nlaunch < 2 || !(side = side_streams_for_current_device())) return GA_OK;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return GA_ERR_CUDA;
    for (int i = 0; i < kSideStreams; ++i)
      if (cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess) return GA_ERR_CUDA;
    c.dp_mark();
    if (cudaEventRecord(fork, c.s) != cudaSuccess) return GA_ERR_CUDA;
    for (int i = 0; i < kSideStreams; ++i)
      if (cudaStreamWaitEvent(side[i], fork, 0) != cudaSuccess) return GA_ERR_CUDA;
    on = true;
    return GA_OK;
  }
  // Stream of the next launch; brackets it with timing events when in order.
  cudaStream_t launch_begin() {
    if (on) {
      c.count_dp();
      return side[n++ % kSideStreams];
    }
    c.dp_begin();
    return c.s;
  }
  void launch_end() {
    if (!on) c.dp_end();
  }
  int end() {
    if (!on) return GA_OK;
    on = false;
    for (int i = 0; i < kSideStreams; ++i)
      if (cudaEventRecord(join[i], side[i]) != cudaSuccess || cudaStreamWaitEvent(c.s, join[i], 0) != cudaSuccess)
        return GA_ERR_CUDA;
    c.dp_mark();
    return GA_OK;
  }
  ~DpFork() {
    end();
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : join)
      if (e) cudaEventDestroy(e);
  }
};

// One plan of a chunk of pairs in one mode.  nt == 0: pair p = (q_p, t_p);
// nt > 0: pair p = (query q0 + p / nt, target p % nt).  Its device state (the
// (class, bin) ranges, task counters and rerun range in `sm`, the sort
// buffers) is its own, so several plans can be enqueued, read back with one
// synchronisation and launched together; the status word and the cell count
// are the call's.
struct ChunkPlan {
  int mode = 0;
  int64_t npairs = 0, nt = 0, q0 = 0;
  int32_t *scores = nullptr;
  int force_long = 0;
  Small *sm = nullptr;
  int32_t *hist = nullptr, *cursor = nullptr;
  uint32_t *keys = nullptr;
  int4 *info = nullptr;
  int32_t *sorted = nullptr, *rerun = nullptr;
  Readback r{};
  int nlaunch = 0, counter = 0;
  // the long class (warp-per-pair stages)
  int long_cnt = 0, long_grid = 0;
  int64_t long_stride = 0;
  size_t long_smem = 0;
  int2 *long_bnd = nullptr;
};

// Plan and sort kernels of one plan, on the call's stream.
int plan_enqueue(Call &c, const SetView &Q, const SetView &T, ChunkPlan &p) {
  if (p.npairs == 0) return GA_OK;
  if (cudaMemsetAsync(p.hist, 0, sizeof(int32_t) * kNumKeys, c.s) != cudaSuccess) return GA_ERR_CUDA;
  if (cudaMemsetAsync(&p.sm->counters, 0, sizeof(p.sm->counters) + sizeof(p.sm->rerun_range), c.s) !=
      cudaSuccess)
    return GA_ERR_CUDA;
  if (cudaMemsetAsync(&p.sm->rmax_long, 0, sizeof(int32_t), c.s) != cudaSuccess) return GA_ERR_CUDA;

  PlanParams pp{};
  pp.q_off = Q.off;
  pp.t_off = T.off;
  pp.npairs = p.npairs;
  pp.nt = p.nt;
  pp.q0 = p.q0;
  pp.qbad = Q.bad;
  pp.tbad = T.bad;
  pp.A = c.sc.A;
  pp.mode = p.mode;
  pp.alpha = c.sc.alpha;
  pp.beta = c.sc.beta;
  pp.sigma_max = c.sc.smax;
  pp.sigma_min = c.sc.smin;
  pp.dna = c.dna && !p.force_long;
  pp.bins = make_bins();
  pp.scores = p.scores;
  pp.keys = p.keys;
  pp.info = p.info;
  pp.status = &c.small->status;
  pp.cells = &c.small->cells;
  pp.rmax_long = &p.sm->rmax_long;
  const unsigned tb = 256;
  const unsigned nb = (unsigned)((p.npairs + tb - 1) / tb);
  plan_kernel<<<nb, tb, 0, c.s>>>(pp);
  hist_kernel<<<nb, tb, 0, c.s>>>(p.keys, p.npairs, p.hist);
  scan_partials_kernel<<<kScanTiles, kScanTile, 0, c.s>>>(p.hist, p.sm->scan_partials);
  scan_apply_kernel<<<kScanTiles, kScanTile, 0, c.s>>>(p.hist, p.sm->scan_partials, p.cursor, p.sm->ranges);
  scatter_kernel<<<nb, tb, 0, c.s>>>(p.keys, p.npairs, p.cursor, p.sorted);
  c.launches += 5;
  return cudaGetLastError() == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

// Bin populations and longest long-class pair of n plans: one copy each,
// one synchronisation.
int plan_readback(Call &c, ChunkPlan *ps, int n) {
  static_assert(8 * sizeof(Readback) <= 4096, "pinned scratch holds the readbacks of 8 plans");
  Readback *rb = (Readback *)pinned_scratch();
  bool any = false;
  for (int k = 0; k < n; ++k) {
    if (ps[k].npairs == 0) continue;
    if (cudaMemcpyAsync(rb + k, ps[k].sm, sizeof(Readback), cudaMemcpyDeviceToHost, c.s) != cudaSuccess)
      return GA_ERR_CUDA;
    any = true;
  }
  if (any && cudaStreamSynchronize(c.s) != cudaSuccess) return GA_ERR_CUDA;
  for (int k = 0; k < n; ++k)
    if (ps[k].npairs > 0) ps[k].r = rb[k];
  return GA_OK;
}

int plan_bin_count(const ChunkPlan &p, int cls, int bin) {
  const int key = cls * kBins + bin;
  return p.r.ranges[2 * key + 1] - p.r.ranges[2 * key];
}

// Launch count, long-class grid and edge buffer of a read-back plan.  The
// buffer is allocated here, before the fork: the side streams start after it.
int launch_prepare(Call &c, ChunkPlan &p) {
  p.nlaunch = 0;
  p.counter = 0;
  if (p.npairs == 0) return GA_OK;
  p.long_cnt = plan_bin_count(p, kClassLong, 0);
  p.nlaunch = p.long_cnt > 0;
  for (int cls = 0; cls < 2; ++cls)
    for (int bin = 0; bin < kKaNumBins; ++bin) p.nlaunch += plan_bin_count(p, cls, bin) > 0;
  const bool profile = !c.dna;
  p.long_smem = profile ? (size_t)kKbWarps * (size_t)(c.sc.A + 1) * (32 * kKbK) : 0;
  if (p.long_cnt > 0) {
    int occ = 0;
    if (long_packed(c.sc, c.dna))
      occ = p.mode == GA_LOCAL ? blocks_per_sm_kw_local()
          : p.mode == GA_GLOBAL ? blocks_per_sm_kw_global()
                                : blocks_per_sm_kw_semi();
    else if (profile)
      occ = p.mode == GA_LOCAL ? blocks_per_sm_kb_local_prof(p.long_smem)
          : p.mode == GA_GLOBAL ? blocks_per_sm_kb_global_prof(p.long_smem)
                                : blocks_per_sm_kb_semi_prof(p.long_smem);
    else
      occ = p.mode == GA_LOCAL ? blocks_per_sm_kb_local_sel(p.long_smem)
          : p.mode == GA_GLOBAL ? blocks_per_sm_kb_global_sel(p.long_smem)
                                : blocks_per_sm_kb_semi_sel(p.long_smem);
    const int64_t want = (p.long_cnt + kKbWarps - 1) / kKbWarps;
    p.long_grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c.nsm * std::max(occ, 1)));
    p.long_stride = (int64_t)p.r.rmax_long + 128;
    p.long_bnd = c.al.get<int2>((size_t)p.long_grid * kKbWarps * (size_t)p.long_stride);
    if (c.al.failed) return GA_ERR_OOM;
  }
  return GA_OK;
}

// Packed tiles that the batch entry points run with their alternative
// lane-group size (8 lanes x 2K columns for tiles K = 7..11): measured on
// GB300 on 1M mutated DNA pairs of 100..300 residues in all three modes,
// each of these tiles is 0.1..0.5 % faster that way, the wide tiles with
// 32 lanes 1..2.4 % slower.  Plans choose their own (ga_plan_autotune).
constexpr uint32_t kEagerLanesAlt = 0x3eu;
static_assert((kEagerLanesAlt & ~kKaAltTiles) == 0, "only tiles with an alternative");

int plan_occupancy_alt(int mode, int bin) {
  return mode == GA_LOCAL ? blocks_per_sm_ka16alt_local(bin) : mode == GA_GLOBAL ? blocks_per_sm_ka16alt_global(bin)
                                                                                  : blocks_per_sm_ka16alt_semi(bin);
}

cudaError_t plan_launch_ka_alt(int mode, int tile, const KAParams &ka, int grid, cudaStream_t s) {
  return mode == GA_LOCAL ? launch_ka16alt_local(tile, ka, grid, s) : mode == GA_GLOBAL ? launch_ka16alt_global(tile, ka, grid, s)
                                                                                        : launch_ka16alt_semi(tile, ka, grid, s);
}

KAParams make_ka(Call &c, const SetView &Q, const SetView &T, const ChunkPlan &p) {
  KAParams ka{};
  ka.packed_q = Q.packed;
  ka.packed_t = T.packed;
  ka.q_off = Q.off;
  ka.t_off = T.off;
  ka.info = p.info;
  ka.sorted = p.sorted;
  std::memcpy(ka.tables, c.sc.tables, sizeof(ka.tables));
  ka.alpha = c.sc.alpha;
  ka.beta = c.sc.beta;
  ka.sigma_max_pos = std::max(c.sc.smax, 0);
  ka.scores = p.scores;
  ka.rerun_list = p.rerun;
  ka.rerun_count = &p.sm->rerun_range[1];
  ka.nt = p.nt;
  ka.q0 = p.q0;
  return ka;
}

// The inter-sequence launch of one (class, bin) of a plan, if it is populated.
int launch_bin(Call &c, const SetView &Q, const SetView &T, ChunkPlan &p, int cls, int bin, DpFork &fk) {
  if (p.npairs == 0) return GA_OK;
  const int cnt = plan_bin_count(p, cls, bin);
  if (cnt <= 0) return GA_OK;
  (cls == 0 ? c.pairs16 : c.pairs32) += cnt;
  KAParams ka = make_ka(c, Q, T, p);
  ka.range = &p.sm->ranges[2 * (cls * kBins + bin)];
  ka.task_counter = &p.sm->counters[p.counter++];
  const bool alt = cls == 0 && (kEagerLanesAlt >> bin & 1u);
  const int ppt = (cls == 0 ? 2 : 1) * (32 / (alt ? ka_alt_g(bin) : kKaG));
  const int64_t ntasks = (cnt + ppt - 1) / ppt;
  int occ;
  if (alt) {
    occ = plan_occupancy_alt(p.mode, bin);
  } else if (cls == 0) {
    occ = p.mode == GA_LOCAL ? blocks_per_sm_ka16_local(bin)
        : p.mode == GA_GLOBAL ? blocks_per_sm_ka16_global(bin)
                              : blocks_per_sm_ka16_semi(bin);
  } else {
    occ = p.mode == GA_LOCAL ? blocks_per_sm_ka32_local(bin)
        : p.mode == GA_GLOBAL ? blocks_per_sm_ka32_global(bin)
                              : blocks_per_sm_ka32_semi(bin);
  }
  const int64_t want = (ntasks + (kKaThreads / 32) - 1) / (kKaThreads / 32);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c.nsm * std::max(occ, 1)));
  cudaError_t e;
  const cudaStream_t ls = fk.launch_begin();
  if (alt) {
    e = plan_launch_ka_alt(p.mode, bin, ka, grid, ls);
  } else if (cls == 0) {
    e = p.mode == GA_LOCAL ? launch_ka16_local(bin, ka, grid, ls)
      : p.mode == GA_GLOBAL ? launch_ka16_global(bin, ka, grid, ls)
                            : launch_ka16_semi(bin, ka, grid, ls);
  } else {
    e = p.mode == GA_LOCAL ? launch_ka32_local(bin, ka, grid, ls)
      : p.mode == GA_GLOBAL ? launch_ka32_global(bin, ka, grid, ls)
                            : launch_ka32_semi(bin, ka, grid, ls);
  }
  fk.launch_end();
  return e == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

// Long pairs (and every pair of an alphabet of more than 4 symbols) of a plan.
int launch_long(Call &c, const SetView &Q, const SetView &T, ChunkPlan &p, DpFork &fk) {
  if (p.npairs == 0 || p.long_cnt <= 0) return GA_OK;
  const bool profile = !c.dna;
  const bool packed = long_packed(c.sc, c.dna);
  (packed ? c.pairs16 : c.pairs32) += p.long_cnt;
  KBParams kb{};
  kb.packed_q = Q.packed;
  kb.packed_t = T.packed;
  kb.q_codes = Q.codes;
  kb.t_codes = T.codes;
  kb.q_off = Q.off;
  kb.t_off = T.off;
  kb.info = p.info;
  kb.sorted = p.sorted;
  kb.range = &p.sm->ranges[2 * (kClassLong * kBins)];
  kb.task_counter = &p.sm->counters[p.counter++];
  std::memcpy(kb.tables, c.sc.tables, sizeof(kb.tables));
  std::memcpy(kb.sigma, c.sc.mat, sizeof(kb.sigma));
  kb.A = c.sc.A;
  kb.alpha = c.sc.alpha;
  kb.beta = c.sc.beta;
  kb.scores = p.scores;
  kb.bnd = p.long_bnd;
  kb.bnd_stride = p.long_stride;
  kb.nt = p.nt;
  kb.q0 = p.q0;
  cudaError_t e;
  const cudaStream_t ls = fk.launch_begin();
  if (packed)
    e = p.mode == GA_LOCAL ? launch_kw_local(kb, p.long_grid, ls)
      : p.mode == GA_GLOBAL ? launch_kw_global(kb, p.long_grid, ls)
                            : launch_kw_semi(kb, p.long_grid, ls);
  else if (profile)
    e = p.mode == GA_LOCAL ? launch_kb_local_prof(kb, p.long_grid, p.long_smem, ls)
      : p.mode == GA_GLOBAL ? launch_kb_global_prof(kb, p.long_grid, p.long_smem, ls)
                            : launch_kb_semi_prof(kb, p.long_grid, p.long_smem, ls);
  else
    e = p.mode == GA_LOCAL ? launch_kb_local_sel(kb, p.long_grid, p.long_smem, ls)
      : p.mode == GA_GLOBAL ? launch_kb_global_sel(kb, p.long_grid, p.long_smem, ls)
                            : launch_kb_semi_sel(kb, p.long_grid, p.long_smem, ls);
  fk.launch_end();
  return e == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

// DP launches of n read-back plans in one fork / join: the inter-sequence
// bins widest tile first (the plans' bins of one width together), so the
// narrow tiles of every plan fill the tail, then the long classes.
int launch_plans(Call &c, const SetView &Q, const SetView &T, ChunkPlan *ps, int n) {
  int nlaunch = 0;
  for (int k = 0; k < n; ++k) nlaunch += ps[k].nlaunch;
  DpFork fk(c);
  if (int rc = fk.begin(nlaunch)) return rc;
  for (int cls = 1; cls >= 0; --cls)
    for (int bin = kKaNumBins - 1; bin >= 0; --bin)
      for (int k = 0; k < n; ++k)
        if (int rc = launch_bin(c, Q, T, ps[k], cls, bin, fk)) return rc;
  for (int k = 0; k < n; ++k)
    if (int rc = launch_long(c, Q, T, ps[k], fk)) return rc;
  return fk.end();
}

// Exact int32 rerun of local int16 pairs whose running max reached the
// int16 limit (queued by the int16x2 kernels on the device); after the join.
int rerun_enqueue(Call &c, const SetView &Q, const SetView &T, ChunkPlan &p) {
  if (p.npairs == 0 || p.mode != GA_LOCAL || !c.dna) return GA_OK;
  int any16 = 0;
  for (int bin = 0; bin < kKaNumBins; ++bin) any16 |= plan_bin_count(p, 0, bin) > 0;
  if (!any16) return GA_OK;
  range_from_count_kernel<<<1, 1, 0, c.s>>>(&p.sm->rerun_range[1], p.sm->rerun_range);
  count_reruns_kernel<<<1, 1, 0, c.s>>>(p.sm->rerun_range, &c.small->rerun_total);
  KAParams ka = make_ka(c, Q, T, p);
  ka.sorted = p.rerun;
  ka.range = p.sm->rerun_range;
  ka.rerun_list = nullptr;
  ka.rerun_count = nullptr;
  ka.task_counter = &p.sm->counters[p.counter++];
  const int bin = kKaNumBins - 1;
  const int occ = blocks_per_sm_ka32_local(bin);
  c.launches += 2;
  c.dp_begin();
  const cudaError_t e = launch_ka32_local(bin, ka, c.nsm * std::max(occ, 1), c.s);
  c.dp_end();
  return e == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

// Plan, read back, launch and rerun several plans of the same pairs (one per
// mode) as one unit: nothing waits for the host between them.
int run_plans(Call &c, const SetView &Q, const SetView &T, ChunkPlan *ps, int n) {
  int rc;
  for (int k = 0; k < n; ++k)
    if ((rc = plan_enqueue(c, Q, T, ps[k]))) return rc;
  if ((rc = plan_readback(c, ps, n))) return rc;
  for (int k = 0; k < n; ++k)
    if ((rc = launch_prepare(c, ps[k]))) return rc;
  if ((rc = launch_plans(c, Q, T, ps, n))) return rc;
  for (int k = 0; k < n; ++k)
    if ((rc = rerun_enqueue(c, Q, T, ps[k]))) return rc;
  return GA_OK;
}

// Plan, sort and run one chunk of pairs in the call's mode, with the call's
// own plan state.
int run_chunk(Call &c, const SetView &Q, const SetView &T, int64_t npairs, int64_t nt, int64_t q0,
              int32_t *scores, int force_long, uint32_t *keys, int4 *info, int32_t *sorted,
              int32_t *rerun_list) {
  if (npairs == 0) return GA_OK;
  ChunkPlan p;
  p.mode = c.mode;
  p.npairs = npairs;
  p.nt = nt;
  p.q0 = q0;
  p.scores = scores;
  p.force_long = force_long;
  p.sm = c.small;
  p.hist = c.hist;
  p.cursor = c.cursor;
  p.keys = keys;
  p.info = info;
  p.sorted = sorted;
  p.rerun = rerun_list;
  return run_plans(c, Q, T, &p, 1);
}

int finish(Call &c, ga_stats *st, cudaEvent_t e0, cudaEvent_t e1, int64_t pairs) {
  if (!st) return GA_OK;
  Readback *rb = (Readback *)pinned_scratch();
  if (cudaEventRecord(e1, c.s) != cudaSuccess) return GA_ERR_CUDA;
  if (cudaMemcpyAsync(rb, c.small, sizeof(Readback), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
      cudaStreamSynchronize(c.s) != cudaSuccess)
    return GA_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  std::memset(st, 0, sizeof(*st));
  st->cells = (int64_t)rb->cells;
  st->pairs = pairs;
  st->pairs_int16 = c.pairs16;
  st->pairs_int32 = c.pairs32;
  st->pairs_int32_rerun = rb->rerun_total;
  st->kernel_ms = ms;
  st->dp_ms = c.dp_ms();
  st->dp_launches = c.dp_launches;
  st->launches = c.launches;
  st->status = rb->status;
  return GA_OK;
}

struct Events {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool on = false;
  Events(bool want, cudaStream_t s) : on(want) {
    if (on) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
  }
  ~Events() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Independent pairs in one or more modes: both sequence sets are validated
// and packed once, then every mode is planned and aligned on the packed
// copies; the scores of mode k go to scores + k * score_stride.
int batch_modes_impl(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                     const int64_t *t_off, int64_t npairs, const ga_scoring *scoring, const int32_t *modes,
                     int32_t nmodes, int32_t *scores, int64_t score_stride, void *stream, ga_stats *stats,
                     int force_long, KnownRange qr = KnownRange(), KnownRange tr = KnownRange()) {
  if (npairs < 0 || !modes || nmodes < 1 || nmodes > 8) return GA_ERR_ARG;
  for (int k = 0; k < nmodes; ++k)
    if (modes[k] < 0 || modes[k] > 2) return GA_ERR_ARG;
  if (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !scores)) return GA_ERR_ARG;
  if (npairs >= (1ll << 31) - 64) return GA_ERR_ARG;
  Call c((cudaStream_t)stream);
  int rc = check_scoring(scoring, &c.sc);
  if (rc) return rc;
  c.mode = modes[0];
  c.timing = stats != nullptr;
  Events ev(stats != nullptr, c.s);
  if ((rc = setup(c))) return rc;
  SetView Q{q_codes, q_off, nullptr, nullptr}, T{t_codes, t_off, nullptr, nullptr};
  if ((rc = prepare_set(c, q_codes, q_off, npairs, &Q.packed, &Q.bad, &c.small->invalid_q, qr))) return rc;
  if ((rc = prepare_set(c, t_codes, t_off, npairs, &T.packed, &T.bad, &c.small->invalid_t, tr))) return rc;
  // one plan per mode (own sort buffers and plan state), all read back with
  // one synchronisation and launched in one fork / join
  ChunkPlan ps[8];
  for (int k = 0; k < nmodes; ++k) {
    ChunkPlan &p = ps[k];
    p.mode = modes[k];
    p.npairs = npairs;
    p.scores = scores + (size_t)k * (size_t)score_stride;
    p.force_long = force_long;
    p.sm = k == 0 ? c.small : c.al.get<Small>(1);
    p.hist = k == 0 ? c.hist : c.al.get<int32_t>(kNumKeys);
    p.cursor = k == 0 ? c.cursor : c.al.get<int32_t>(kNumKeys);
    p.keys = c.al.get<uint32_t>((size_t)npairs);
    p.info = c.al.get<int4>((size_t)npairs);
    p.sorted = c.al.get<int32_t>((size_t)npairs);
    p.rerun = c.al.get<int32_t>((size_t)npairs);
    if (c.al.failed) return GA_ERR_OOM;
    if (k > 0 && cudaMemsetAsync(p.sm, 0, sizeof(Small), c.s) != cudaSuccess) return GA_ERR_CUDA;
  }
  if ((rc = run_plans(c, Q, T, ps, nmodes))) return rc;
  return finish(c, stats, ev.e0, ev.e1, npairs * nmodes);
}

int batch_impl(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
               const int64_t *t_off, int64_t npairs, const ga_scoring *scoring, int32_t mode,
               int32_t *scores, void *stream, ga_stats *stats, int force_long,
               KnownRange qr = KnownRange(), KnownRange tr = KnownRange()) {
  return batch_modes_impl(q_codes, q_off, t_codes, t_off, npairs, scoring, &mode, 1, scores, 0, stream, stats,
                          force_long, qr, tr);
}

__global__ void fill_i32_kernel(int32_t *p, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Bracket of the minimal certified width from the doubling result w (w_used
// of a doubling run that started at 0): w = 0 or 1 is exact, otherwise the
// width w/2 failed, so w_min lies in [w/2 + 1, min(w, min(m, n))] (a band of
// half-width min(m, n) covers the matrix).  Invalid pairs (w < 0) are done.
__global__ void bisect_init_kernel(const int64_t *q_off, const int64_t *t_off, int64_t npairs,
                                   const int32_t *w_used, int32_t *lo, int32_t *hi, int32_t *maxgap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int gap = 0;
  if (i < npairs) {
    const int w = w_used[i];
    const int64_t m = q_off[i + 1] - q_off[i], n = t_off[i + 1] - t_off[i];
    const int cap = (int)(m < n ? m : n);
    int l = w, h = w;
    if (w < 0) {
      l = h = -1;
    } else if (w >= 2) {
      h = w < cap ? w : cap;
      l = w / 2 + 1 < h ? w / 2 + 1 : h;
    }
    lo[i] = l;
    hi[i] = h;
    gap = h - l;
  }
  gap = __reduce_max_sync(0xffffffffu, (unsigned)gap);
  if ((threadIdx.x & 31) == 0 && gap > 0) atomicMax(maxgap, gap);
}

__global__ void bisect_final_kernel(int64_t npairs, const int32_t *lo, int32_t *w_min) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npairs) w_min[i] = lo[i];
}

// A planned banded run (global mode, alphabets of <= 4 symbols): both sets
// packed, pairs ordered by estimated band work, boundary buffers sized.
struct BandRun {
  Call &c;
  SetView Q, T;
  int64_t npairs;
  uint32_t *keys = nullptr;
  int32_t *sorted = nullptr;
  int max_rows = 0, grid = 0, launches = 0;
  bool packed = false;  // packed int16x2 kernel (sigma_max + alpha <= kKzMaxStep)
  int64_t stride = 0;
  int2 *bnd = nullptr;
  BandRun(Call &cc, const uint8_t *qc, const int64_t *qo, const uint8_t *tc, const int64_t *to, int64_t np)
      : c(cc), Q{qc, qo, nullptr, nullptr}, T{tc, to, nullptr, nullptr}, npairs(np) {}

  int prepare() {
    int rc;
    if ((rc = prepare_set(c, Q.codes, Q.off, npairs, &Q.packed, &Q.bad, &c.small->invalid_q))) return rc;
    if ((rc = prepare_set(c, T.codes, T.off, npairs, &T.packed, &T.bad, &c.small->invalid_t))) return rc;
    keys = c.al.get<uint32_t>((size_t)npairs);
    sorted = c.al.get<int32_t>((size_t)npairs);
    return c.al.failed ? GA_ERR_OOM : GA_OK;
  }

  // Validity, closed forms of empty pairs, work keys and the sorted order.
  int plan(const int32_t *w0, int32_t default_w0, int32_t *scores, int32_t *w_used) {
    if (cudaMemsetAsync(c.hist, 0, sizeof(int32_t) * kNumKeys, c.s) != cudaSuccess) return GA_ERR_CUDA;
    BandPlanParams bp{};
    bp.q_off = Q.off;
    bp.t_off = T.off;
    bp.npairs = npairs;
    bp.qbad = Q.bad;
    bp.tbad = T.bad;
    bp.w0 = w0;
    bp.default_w0 = default_w0;
    bp.alpha = c.sc.alpha;
    bp.beta = c.sc.beta;
    bp.scores = scores;
    bp.w_used = w_used;
    bp.keys = keys;
    bp.status = &c.small->status;
    bp.cells = &c.small->cells;
    bp.max_rows = &c.small->max_rows;
    bp.max_span = &c.small->max_band_span;
    bp.stage_cols = kBandStageCols;
    const unsigned nb = (unsigned)((npairs + 255) / 256);
    band_plan_kernel<<<nb, 256, 0, c.s>>>(bp);
    hist_kernel<<<nb, 256, 0, c.s>>>(keys, npairs, c.hist);
    scan_partials_kernel<<<kScanTiles, kScanTile, 0, c.s>>>(c.hist, c.small->scan_partials);
    scan_apply_kernel<<<kScanTiles, kScanTile, 0, c.s>>>(c.hist, c.small->scan_partials, c.cursor,
                                                         c.small->ranges);
    scatter_kernel<<<nb, 256, 0, c.s>>>(keys, npairs, c.cursor, sorted);
    c.launches += 5;
    if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;
    int32_t *h = (int32_t *)pinned_scratch();
    if (cudaMemcpyAsync(h, &c.small->max_rows, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaStreamSynchronize(c.s) != cudaSuccess)
      return GA_ERR_CUDA;
    max_rows = h[0];
    if (max_rows > 0) {
      // the packed kernel numbers its iterations in int32: a pair runs at
      // most max(m + 1, 128) x super-stages + m + 64 of them; calls with
      // larger pairs take the int32 kernel, which runs one stage at a time
      packed = std::max(c.sc.smax, 0) + c.sc.alpha <= kKzMaxStep && h[1] < kKzMaxSpan;
      const int occ = std::max(packed ? blocks_per_sm_kz() : blocks_per_sm_kc(), 1);
      const int64_t want = (npairs + kKcWarps - 1) / kKcWarps;
      grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c.nsm * occ));
      stride = (int64_t)max_rows + 128;
      // edge buffers, one per warp: int2 per row (kc_kernel), KZEdge (16
      // bytes) per row (kz_kernel)
      const size_t rows = (size_t)grid * kKcWarps * (size_t)stride;
      bnd = packed ? reinterpret_cast<int2 *>(c.al.get<int4>(rows)) : c.al.get<int2>(rows);
      if (c.al.failed) return GA_ERR_OOM;
    }
    return GA_OK;
  }

  // One launch of the banded kernel over the planned order: band doubling
  // (bis_lo == nullptr) or one bisection step.  Each launch takes a fresh
  // task counter.
  int launch(const int32_t *w0, int32_t default_w0, int32_t *scores, int32_t *w_used, int32_t *bis_lo,
             int32_t *bis_hi) {
    if (max_rows <= 0) return GA_OK;
    if (launches >= 62) return GA_ERR_ARG;
    KCParams kc{};
    kc.packed_q = Q.packed;
    kc.packed_t = T.packed;
    kc.q_off = Q.off;
    kc.t_off = T.off;
    kc.order = sorted;
    kc.range = c.small->ranges;  // class 0, bin 0: every non-trivial pair
    kc.task_counter = &c.small->counters[launches++];
    std::memcpy(kc.tables, c.sc.tables, sizeof(kc.tables));
    kc.alpha = c.sc.alpha;
    kc.beta = c.sc.beta;
    kc.sigma_max_pos = std::max(c.sc.smax, 0);
    kc.w0 = w0;
    kc.default_w0 = default_w0;
    kc.scores = scores;
    kc.w_used = w_used;
    kc.retries = &c.small->band_retries;
    kc.cells = &c.small->band_cells;
    kc.bnd = bnd;
    kc.bnd_stride = stride;
    kc.bis_lo = bis_lo;
    kc.bis_hi = bis_hi;
    c.dp_begin();
    const cudaError_t e = packed ? launch_kz(kc, grid, c.s) : launch_kc(kc, grid, c.s);
    c.dp_end();
    return e == cudaSuccess ? GA_OK : GA_ERR_CUDA;
  }

  int band_stats(ga_stats *st) {
    unsigned long long *hb = (unsigned long long *)pinned_scratch();
    if (cudaMemcpyAsync(hb, &c.small->band_retries, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaStreamSynchronize(c.s) != cudaSuccess)
      return GA_ERR_CUDA;
    st->band_retries = (int64_t)hb[0];
    st->banded_cells = (int64_t)hb[1];
    return GA_OK;
  }
};

// Features (predict == false) or fused prediction of DNA pairs.
int features_impl(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                  const int64_t *t_off, int64_t npairs, float *features, const uint16_t *wb,
                  float margin, int32_t *w0, float *y, void *stream, ga_stats *stats) {
  if (npairs >= (1ll << 31) - 64) return GA_ERR_ARG;
  Call c((cudaStream_t)stream);
  c.sc.A = 4;  // DNA codes 0..3; residues are validated while packing
  c.mode = GA_GLOBAL;
  c.timing = stats != nullptr;
  Events ev(stats != nullptr, c.s);
  int rc;
  if ((rc = setup(c))) return rc;
  if (npairs == 0) return finish(c, stats, ev.e0, ev.e1, 0);
  SetView Q{q_codes, q_off, nullptr, nullptr}, T{t_codes, t_off, nullptr, nullptr};
  if ((rc = prepare_set(c, q_codes, q_off, npairs, &Q.packed, &Q.bad, &c.small->invalid_q))) return rc;
  if ((rc = prepare_set(c, t_codes, t_off, npairs, &T.packed, &T.bad, &c.small->invalid_t))) return rc;
  BandFeatParams fp{};
  fp.packed_q = Q.packed;
  fp.packed_t = T.packed;
  fp.q_off = q_off;
  fp.t_off = t_off;
  fp.qbad = Q.bad;
  fp.tbad = T.bad;
  fp.npairs = npairs;
  fp.features = features;
  fp.wb = wb;
  fp.margin = margin;
  fp.y = y;
  fp.w0 = w0;
  fp.status = &c.small->status;
  const size_t smem = feat_smem_bytes(wb != nullptr);
  const bool attr_ok =  // per call: the attribute belongs to the current device
      cudaFuncSetAttribute(band_features_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)feat_smem_bytes(true)) == cudaSuccess &&
      cudaFuncSetAttribute(band_features_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)feat_smem_bytes(false)) == cudaSuccess;
  if (!attr_ok) return GA_ERR_CUDA;
  const int grid = (int)std::min<int64_t>(npairs, (int64_t)c.nsm * 4);
  if (wb)
    band_features_kernel<true><<<grid, kFeatThreads, smem, c.s>>>(fp);
  else
    band_features_kernel<false><<<grid, kFeatThreads, smem, c.s>>>(fp);
  ++c.launches;
  if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;
  return finish(c, stats, ev.e0, ev.e1, npairs);
}

// Database search of protein (alphabets of > 4 symbols), local mode, on the
// packed query-profile kernel: targets sorted longest first, queries binned
// by length (columns per lane K = 8, 16, 24 or 32; longer queries run in
// stages of 512 columns), flagged pairs recomputed exactly in int32.
template <int K>
int launch_kp(Call &c, KPParams &kp, int64_t max_grid) {
  const size_t smem = sizeof(uint32_t) * (size_t)kp_prof_words<K>(c.sc.A);
  if (cudaFuncSetAttribute(kp_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GA_ERR_CUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kp_kernel<K>, 32 * kKpWarps, smem) != cudaSuccess)
    return GA_ERR_CUDA;
  const int64_t ntasks = (int64_t)((kp.nqb + 1) / 2) * ((kp.ntv + kKpGroups - 1) / kKpGroups);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>({ntasks, (int64_t)c.nsm * std::max(occ, 1), max_grid}));
  c.dp_begin();
  kp_kernel<K><<<grid, 32 * kKpWarps, smem, c.s>>>(kp);
  c.dp_end();
  return cudaGetLastError() == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

// Tiles of the protein search: columns per lane K (16K columns per group)
// and the measured relative rate of the kernel per computed cell on GB300
// (wider tiles amortise the per-row work over more columns); a query of
// several stages pays for its profile rebuilds and stage edges.
constexpr int kKpTiles = 6;
constexpr int kKpTileK[kKpTiles] = {8, 16, 20, 24, 28, 32};
constexpr double kKpRate[kKpTiles] = {0.81, 0.92, 0.96, 1.0, 1.08, 1.02};
constexpr double kKpStagedRate = 0.97;

// Tile of a query of m columns: the one that minimises the estimated time
// ceil(m / 16K) * 16K / rate(K).
int kp_bin_for(int64_t m) {
  int best = kKpTiles - 1;
  double tbest = 1e300;
  for (int b = 0; b < kKpTiles; ++b) {
    const int64_t w = (int64_t)kKpG * kKpTileK[b];
    const int64_t nst = (m + w - 1) / w;
    const double t = (double)(nst * w) / (kKpRate[b] * (nst > 1 ? kKpStagedRate : 1.0));
    if (t < tbest) {
      tbest = t;
      best = b;
    }
  }
  return best;
}

int launch_kp_tile(Call &c, KPParams &kp, int64_t max_grid, int b) {
  switch (kKpTileK[b]) {
    case 8: return launch_kp<8>(c, kp, max_grid);
    case 16: return launch_kp<16>(c, kp, max_grid);
    case 20: return launch_kp<20>(c, kp, max_grid);
    case 24: return launch_kp<24>(c, kp, max_grid);
    case 28: return launch_kp<28>(c, kp, max_grid);
    default: return launch_kp<32>(c, kp, max_grid);
  }
}

int cross_protein_local(Call &c, const uint8_t *q_codes, const int64_t *q_off, int64_t nq,
                        const uint8_t *t_codes, const int64_t *t_off, int64_t nt, int32_t *scores,
                        ga_stats *stats, cudaEvent_t e0, cudaEvent_t e1) {
  int rc;
  SetView Q{q_codes, q_off, nullptr, nullptr}, T{t_codes, t_off, nullptr, nullptr};
  if ((rc = prepare_set(c, q_codes, q_off, nq, &Q.packed, &Q.bad, &c.small->invalid_q))) return rc;
  uint32_t *t_packed5 = nullptr;
  if ((rc = prepare_set(c, t_codes, t_off, nt, &T.packed, &T.bad, &c.small->invalid_t, KnownRange(), &t_packed5)))
    return rc;
  if (nt >= (1ll << 31) - 64 || nq * nt >= (1ll << 31) - 64) return GA_ERR_ARG;
  uint32_t *keys = c.al.get<uint32_t>((size_t)nt);
  int32_t *sorted = c.al.get<int32_t>((size_t)nt);
  // flagged pairs are rerun in int32 one list at a time; a search with more
  // of them than the list holds finds the rest by scanning for their marks
  const int32_t rerun_cap = (int32_t)std::min<int64_t>(std::max<int64_t>(nq * nt, 1), 1 << 16);
  int32_t *rerun = c.al.get<int32_t>((size_t)rerun_cap);
  if (c.al.failed) return GA_ERR_OOM;
  // targets: longest first, invalid ones left out
  if (cudaMemsetAsync(c.hist, 0, sizeof(int32_t) * kNumKeys, c.s) != cudaSuccess) return GA_ERR_CUDA;
  const unsigned nbt = (unsigned)((nt + 255) / 256);
  kp_target_keys_kernel<<<nbt, 256, 0, c.s>>>(t_off, nt, T.bad, keys, &c.small->max_rows);
  hist_kernel<<<nbt, 256, 0, c.s>>>(keys, nt, c.hist);
  scan_partials_kernel<<<kScanTiles, kScanTile, 0, c.s>>>(c.hist, c.small->scan_partials);
  scan_apply_kernel<<<kScanTiles, kScanTile, 0, c.s>>>(c.hist, c.small->scan_partials, c.cursor, c.small->ranges);
  scatter_kernel<<<nbt, 256, 0, c.s>>>(keys, nt, c.cursor, sorted);
  c.launches += 5;
  if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;
  // host view: query offsets and validity, target count and longest target
  std::vector<int64_t> hqo((size_t)nq + 1);
  std::vector<uint8_t> hqb((size_t)nq);
  Small *hs = (Small *)pinned_scratch();
  static_assert(sizeof(Small) <= 4096, "pinned scratch holds the call's scalars");
  if (cudaMemcpyAsync(hqo.data(), q_off, sizeof(int64_t) * (size_t)(nq + 1), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
      cudaMemcpyAsync(hqb.data(), Q.bad, (size_t)nq, cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
      cudaMemcpyAsync(hs, c.small, sizeof(Small), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
      cudaStreamSynchronize(c.s) != cudaSuccess)
    return GA_ERR_CUDA;
  const int32_t ntv = hs->ranges[1] - hs->ranges[0];
  const int32_t max_len = hs->max_rows;
  bool any_bad = ntv < nt;
  for (int64_t k = 0; k < nq; ++k) any_bad |= hqb[k] != 0;
  if (any_bad) {
    kp_invalid_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nq * nt + 255) / 256, (int64_t)c.nsm * 32)),
                        256, 0, c.s>>>(Q.bad, nq, T.bad, nt, scores, &c.small->status);
    ++c.launches;
  }
  // query bins: one tile per query (kp_bin_for)
  std::vector<int32_t> bins[kKpTiles];
  int64_t cells = 0, tcells = 0;
  for (int64_t k = 0; k < nq; ++k) {
    if (hqb[k]) continue;
    const int64_t m = hqo[k + 1] - hqo[k];
    bins[kp_bin_for(m)].push_back((int32_t)k);
    cells += m;
  }
  // the kernel packs queries 2i and 2i+1 of a bin into one register; sorted
  // by length, the two queries of a pair have the same number of stages
  for (auto &b : bins)
    std::stable_sort(b.begin(), b.end(), [&](int32_t x, int32_t y) {
      return hqo[(size_t)x + 1] - hqo[(size_t)x] > hqo[(size_t)y + 1] - hqo[(size_t)y];
    });
  {
    std::vector<int64_t> hto((size_t)nt + 1);
    std::vector<uint8_t> htb((size_t)nt);
    if (cudaMemcpy(hto.data(), t_off, sizeof(int64_t) * (size_t)(nt + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(htb.data(), T.bad, (size_t)nt, cudaMemcpyDeviceToHost) != cudaSuccess)
      return GA_ERR_CUDA;
    for (int64_t l = 0; l < nt; ++l)
      if (!htb[l]) tcells += hto[l + 1] - hto[l];
  }
  cells *= tcells;
  int32_t *dq = c.al.get<int32_t>((size_t)std::max<int64_t>(nq, 1));
  if (c.al.failed) return GA_ERR_OOM;
  std::vector<int32_t> flat;
  for (int b = 0; b < kKpTiles; ++b) flat.insert(flat.end(), bins[b].begin(), bins[b].end());
  if (!flat.empty() &&
      cudaMemcpyAsync(dq, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice, c.s) != cudaSuccess)
    return GA_ERR_CUDA;
  // per-group stage edges: every group slot of the largest grid
  const int64_t max_grid = (int64_t)c.nsm * 4;
  const int64_t stride = (int64_t)std::max(max_len, 0) + 64;
  int2 *bnd = c.al.get<int2>((size_t)max_grid * kKpGroups * (size_t)stride);
  if (c.al.failed) return GA_ERR_OOM;
  KPParams kp{};
  kp.q_codes = q_codes;
  kp.q_off = q_off;
  kp.t_codes = t_codes;
  kp.t_packed5 = t_packed5;
  kp.t_off = t_off;
  kp.t_sorted = sorted;
  kp.ntv = ntv;
  kp.nt = nt;
  kp.A = c.sc.A;
  kp.alpha = c.sc.alpha;
  kp.beta = c.sc.beta;
  kp.sigma_max_pos = std::max(c.sc.smax, 0);
  std::memcpy(kp.sigma, c.sc.mat, sizeof(kp.sigma));
  kp.scores = scores;
  kp.rerun_list = rerun;
  kp.rerun_count = &c.small->rerun_range[1];
  kp.rerun_cap = rerun_cap;
  kp.bnd = bnd;
  kp.bnd_stride = stride;
  size_t off = 0;
  for (int b = 0; b < kKpTiles; ++b) {
    if (bins[b].empty() || ntv == 0) {
      off += bins[b].size();
      continue;
    }
    kp.queries = dq + off;
    kp.nqb = (int32_t)bins[b].size();
    kp.task_counter = &c.small->counters[b];
    off += bins[b].size();
    rc = launch_kp_tile(c, kp, max_grid, b);
    if (rc) return rc;
  }
  // exact int32 rerun of flagged pairs (rare: a local score near 32767).
  // Each pass reruns the pairs of the list; when the kernels flagged more
  // pairs than the list holds, the next list is collected from the marks
  // left in the scores (a rerun overwrites its pair's mark).
  int32_t *hn = (int32_t *)pinned_scratch();
  if (cudaMemcpyAsync(hn, &c.small->rerun_range[1], sizeof(int32_t), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
      cudaStreamSynchronize(c.s) != cudaSuccess)
    return GA_ERR_CUDA;
  const int32_t nre = hn[0];
  int32_t pending = nre;
  bool from_list = true;
  int64_t *info = nre > 0 ? c.al.get<int64_t>((size_t)std::min(nre, rerun_cap) * 4) : nullptr;
  if (c.al.failed) return GA_ERR_OOM;
  std::vector<int32_t> ids;
  std::vector<int64_t> hinfo;
  while (pending > 0) {
    if (!from_list) {  // collect the next list from the marks
      if (cudaMemsetAsync(&c.small->rerun_range[1], 0, sizeof(int32_t), c.s) != cudaSuccess) return GA_ERR_CUDA;
      const int64_t total = nq * nt;
      kp_collect_marked_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256,
                                                                                  (int64_t)c.nsm * 32)),
                                 256, 0, c.s>>>(scores, total, rerun, rerun_cap, &c.small->rerun_range[1]);
      ++c.launches;
      if (cudaMemcpyAsync(hn, &c.small->rerun_range[1], sizeof(int32_t), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
          cudaStreamSynchronize(c.s) != cudaSuccess)
        return GA_ERR_CUDA;
      pending = hn[0];
      if (pending <= 0) break;
    }
    const int32_t n_now = std::min(pending, rerun_cap);
    ids.resize((size_t)n_now);
    hinfo.resize((size_t)n_now * 4);
    kp_rerun_info_kernel<<<(unsigned)((n_now + 255) / 256), 256, 0, c.s>>>(rerun, n_now, nt, q_off, t_off, info);
    ++c.launches;
    if (cudaMemcpyAsync(ids.data(), rerun, sizeof(int32_t) * (size_t)n_now, cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaMemcpyAsync(hinfo.data(), info, sizeof(int64_t) * (size_t)n_now * 4, cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaStreamSynchronize(c.s) != cudaSuccess)
      return GA_ERR_CUDA;
    for (int32_t i = 0; i < n_now; ++i) {
      const int64_t *f = &hinfo[(size_t)i * 4];
      rc = sv_align_pair(q_codes + f[0], f[1], t_codes + f[2], f[3], c.sc.A, c.sc.mat, c.sc.alpha, c.sc.beta,
                         GA_LOCAL, scores + ids[i], c.s, nullptr);
      if (rc) return rc;
    }
    c.pairs32 += n_now;
    pending = (from_list && pending <= rerun_cap) ? 0 : 1;  // an overflowed list: rescan
    from_list = false;
  }
  c.pairs16 += (int64_t)flat.size() * ntv - nre;
  rc = finish(c, stats, e0, e1, nq * nt);
  if (!rc && stats) {
    stats->cells = cells;
    stats->pairs_int32_rerun = nre;
  }
  return rc;
}


// ---- batch plans (include/gotoh_plan.h) ---------------------------------
// The workspace of a batch is allocated once; a run enqueues the same
// kernels as ga_align_batch, but with every size that batch_impl reads back
// from the device (the residue range of each set, the bin populations, the
// longest long-class pair) replaced by the plan's capacity, so nothing in a
// run waits for the host and the whole run can be captured in a graph.

constexpr int kPlanSide = 4;  // side streams for concurrent bins
static_assert(GA_TILE_COUNT == kKaNumBins, "one tuning bit per inter-sequence tile");
static_assert(GA_TILE_ALT_MASK == kKaAltTiles, "the header lists the tiles with an alternative lane-group size");

struct PlanImpl {
  int dev = 0, nsm = 0, mode = 0;
  Scoring sc;
  int64_t max_pairs = 0, max_res = 0;
  int32_t max_len = 0;
  ga_tuning tune{};
  int occ16[kKaNumBins] = {}, occ32[kKaNumBins] = {}, occ16alt[kKaNumBins] = {};
  int occ_kb = 0, long_grid = 0;
  bool long_packed = false;
  size_t long_smem = 0;
  Small *small = nullptr;
  int32_t *hist = nullptr, *cursor = nullptr;
  uint32_t *packed_q = nullptr, *packed_t = nullptr;
  uint8_t *qbad = nullptr, *tbad = nullptr;
  uint32_t *keys = nullptr;
  int4 *info = nullptr;
  int32_t *sorted = nullptr, *rerun = nullptr;
  int2 *bnd = nullptr;
  int64_t bnd_stride = 0;
  std::vector<void *> allocs;
  cudaStream_t side[kPlanSide] = {};
  cudaEvent_t fork = nullptr, join[kPlanSide] = {};
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;

  template <class T>
  T *alloc(size_t n) {
    void *p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T) + 256) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return (T *)p;
  }
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  ~PlanImpl() {
    drop_graph();
    for (void *p : allocs) cudaFree(p);
    for (int i = 0; i < kPlanSide; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

int plan_occupancy(int cls, int mode, int bin) {
  if (cls == 0)
    return mode == GA_LOCAL ? blocks_per_sm_ka16_local(bin) : mode == GA_GLOBAL ? blocks_per_sm_ka16_global(bin)
                                                                                : blocks_per_sm_ka16_semi(bin);
  return mode == GA_LOCAL ? blocks_per_sm_ka32_local(bin) : mode == GA_GLOBAL ? blocks_per_sm_ka32_global(bin)
                                                                              : blocks_per_sm_ka32_semi(bin);
}

cudaError_t plan_launch_ka(int cls, int mode, int tile, const KAParams &ka, int grid, cudaStream_t s) {
  if (cls == 0)
    return mode == GA_LOCAL ? launch_ka16_local(tile, ka, grid, s) : mode == GA_GLOBAL ? launch_ka16_global(tile, ka, grid, s)
                                                                                       : launch_ka16_semi(tile, ka, grid, s);
  return mode == GA_LOCAL ? launch_ka32_local(tile, ka, grid, s) : mode == GA_GLOBAL ? launch_ka32_global(tile, ka, grid, s)
                                                                                     : launch_ka32_semi(tile, ka, grid, s);
}

int plan_create(const ga_scoring *scoring, int32_t mode, int64_t max_pairs, int64_t max_res, int32_t max_len,
                PlanImpl **out) {
  if (!out || mode < 0 || mode > 2 || max_pairs < 1 || max_pairs >= (1ll << 31) - 64 || max_res < 0 ||
      max_len < 1 || max_len > (1 << 24))
    return GA_ERR_ARG;
  std::unique_ptr<PlanImpl> P(new PlanImpl());
  int rc = check_scoring(scoring, &P->sc);
  if (rc) return rc;
  P->mode = mode;
  P->max_pairs = max_pairs;
  P->max_res = max_res;
  P->max_len = max_len;
  P->tune.tiles16 = P->tune.tiles32 = (1u << kKaNumBins) - 1;
  P->tune.concurrent = 0;
  if (cudaGetDevice(&P->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, P->dev) != cudaSuccess)
    return GA_ERR_CUDA;
  const bool dna = P->sc.A <= 4;
  for (int b = 0; b < kKaNumBins; ++b) {
    P->occ16[b] = std::max(plan_occupancy(0, mode, b), 1);
    P->occ32[b] = std::max(plan_occupancy(1, mode, b), 1);
    if (kKaAltTiles >> b & 1u) P->occ16alt[b] = std::max(plan_occupancy_alt(mode, b), 1);
  }
  P->long_smem = dna ? 0 : (size_t)kKbWarps * (size_t)(P->sc.A + 1) * (32 * kKbK);
  P->long_packed = long_packed(P->sc, dna);
  P->occ_kb = P->long_packed ? (mode == GA_LOCAL ? blocks_per_sm_kw_local() : mode == GA_GLOBAL ? blocks_per_sm_kw_global()
                                                                                            : blocks_per_sm_kw_semi())
            : dna ? (mode == GA_LOCAL ? blocks_per_sm_kb_local_sel(0) : mode == GA_GLOBAL ? blocks_per_sm_kb_global_sel(0)
                                                                                         : blocks_per_sm_kb_semi_sel(0))
                  : (mode == GA_LOCAL ? blocks_per_sm_kb_local_prof(P->long_smem)
                                      : mode == GA_GLOBAL ? blocks_per_sm_kb_global_prof(P->long_smem)
                                                          : blocks_per_sm_kb_semi_prof(P->long_smem));
  P->occ_kb = std::max(P->occ_kb, 1);
  P->long_grid = (int)std::min<int64_t>((int64_t)P->nsm * P->occ_kb, (max_pairs + kKbWarps - 1) / kKbWarps);
  P->bnd_stride = (int64_t)max_len + 128;
  P->small = P->alloc<Small>(1);
  P->hist = P->alloc<int32_t>(kNumKeys);
  P->cursor = P->alloc<int32_t>(kNumKeys);
  if (dna) {
    P->packed_q = P->alloc<uint32_t>((size_t)(max_res / 16 + 2));
    P->packed_t = P->alloc<uint32_t>((size_t)(max_res / 16 + 2));
  }
  P->qbad = P->alloc<uint8_t>((size_t)max_pairs + 1);
  P->tbad = P->alloc<uint8_t>((size_t)max_pairs + 1);
  P->keys = P->alloc<uint32_t>((size_t)max_pairs);
  P->info = P->alloc<int4>((size_t)max_pairs);
  P->sorted = P->alloc<int32_t>((size_t)max_pairs);
  P->rerun = P->alloc<int32_t>((size_t)max_pairs);
  P->bnd = P->alloc<int2>((size_t)P->long_grid * kKbWarps * (size_t)P->bnd_stride);
  if (!P->small || !P->hist || !P->cursor || !P->qbad || !P->tbad || !P->keys || !P->info || !P->sorted ||
      !P->rerun || !P->bnd || (dna && (!P->packed_q || !P->packed_t)))
    return GA_ERR_OOM;
  for (int i = 0; i < kPlanSide; ++i)
    if (cudaStreamCreateWithFlags(&P->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->join[i], cudaEventDisableTiming) != cudaSuccess)
      return GA_ERR_CUDA;
  if (cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return GA_ERR_CUDA;
  *out = P.release();
  return GA_OK;
}

// One run, enqueued on s with no host synchronisation and no allocation.
int plan_enqueue(PlanImpl &P, const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                 const int64_t *t_off, int64_t npairs, int32_t *scores, cudaStream_t s) {
  if (npairs < 0 || npairs > P.max_pairs) return GA_ERR_ARG;
  if (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !scores)) return GA_ERR_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != P.dev) return GA_ERR_ARG;
  if (cudaMemsetAsync(P.small, 0, sizeof(Small), s) != cudaSuccess ||
      cudaMemsetAsync(P.hist, 0, sizeof(int32_t) * kNumKeys, s) != cudaSuccess)
    return GA_ERR_CUDA;
  if (npairs == 0) return GA_OK;
  const int A = P.sc.A;
  const bool dna = A <= 4;
  const unsigned vb = (unsigned)((npairs + 255) / 256);
  const unsigned pb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((P.max_res / 16 + 256) / 256, (int64_t)P.nsm * 16));
  plan_pack_kernel<<<pb, 256, 0, s>>>(q_codes, q_off, npairs, P.max_res, A, P.packed_q, &P.small->invalid_q);
  plan_pack_kernel<<<pb, 256, 0, s>>>(t_codes, t_off, npairs, P.max_res, A, P.packed_t, &P.small->invalid_t);
  plan_validate_kernel<<<vb, 256, 0, s>>>(q_codes, q_off, npairs, P.max_res, P.max_len, A, &P.small->invalid_q, P.qbad);
  plan_validate_kernel<<<vb, 256, 0, s>>>(t_codes, t_off, npairs, P.max_res, P.max_len, A, &P.small->invalid_t, P.tbad);

  // bins: the active tiles, narrowest first
  int tile16[kKaNumBins], tile32[kKaNumBins], n16 = 0, n32 = 0;
  for (int b = 0; b < kKaNumBins; ++b) {
    if (P.tune.tiles16 >> b & 1u) tile16[n16++] = b;
    if (P.tune.tiles32 >> b & 1u) tile32[n32++] = b;
  }
  PlanParams pp{};
  pp.q_off = q_off;
  pp.t_off = t_off;
  pp.npairs = npairs;
  pp.qbad = P.qbad;
  pp.tbad = P.tbad;
  pp.A = A;
  pp.mode = P.mode;
  pp.alpha = P.sc.alpha;
  pp.beta = P.sc.beta;
  pp.sigma_max = P.sc.smax;
  pp.sigma_min = P.sc.smin;
  pp.dna = dna;
  pp.bins.n16 = n16;
  pp.bins.n32 = n32;
  for (int i = 0; i < n16; ++i) pp.bins.w16[i] = kKaG * kKaK[tile16[i]];
  for (int i = 0; i < n32; ++i) pp.bins.w32[i] = kKaG * kKaK[tile32[i]];
  pp.scores = scores;
  pp.keys = P.keys;
  pp.info = P.info;
  pp.status = &P.small->status;
  pp.cells = &P.small->cells;
  pp.rmax_long = &P.small->rmax_long;
  plan_kernel<<<vb, 256, 0, s>>>(pp);
  hist_kernel<<<vb, 256, 0, s>>>(P.keys, npairs, P.hist);
  scan_partials_kernel<<<kScanTiles, kScanTile, 0, s>>>(P.hist, P.small->scan_partials);
  scan_apply_kernel<<<kScanTiles, kScanTile, 0, s>>>(P.hist, P.small->scan_partials, P.cursor, P.small->ranges);
  scatter_kernel<<<vb, 256, 0, s>>>(P.keys, npairs, P.cursor, P.sorted);
  if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;

  KAParams ka{};
  ka.packed_q = P.packed_q;
  ka.packed_t = P.packed_t;
  ka.q_off = q_off;
  ka.t_off = t_off;
  ka.info = P.info;
  ka.sorted = P.sorted;
  std::memcpy(ka.tables, P.sc.tables, sizeof(ka.tables));
  ka.alpha = P.sc.alpha;
  ka.beta = P.sc.beta;
  ka.sigma_max_pos = std::max(P.sc.smax, 0);
  ka.scores = scores;
  ka.rerun_list = P.rerun;
  ka.rerun_count = &P.small->rerun_range[1];

  // every bin (widest first) plus the long class, one persistent launch
  // each; concurrent: round-robin over the side streams, joined on s
  const bool conc = P.tune.concurrent != 0;
  int nlaunch = 0, counter = 0;
  auto stream_for = [&](int i) { return conc ? P.side[i % kPlanSide] : s; };
  if (conc) {
    if (cudaEventRecord(P.fork, s) != cudaSuccess) return GA_ERR_CUDA;
    for (int i = 0; i < kPlanSide; ++i)
      if (cudaStreamWaitEvent(P.side[i], P.fork, 0) != cudaSuccess) return GA_ERR_CUDA;
  }
  if (dna) {
    for (int cls = 0; cls < 2; ++cls) {
      const int nb = cls == 0 ? n16 : n32;
      for (int i = nb - 1; i >= 0; --i) {
        const int tile = cls == 0 ? tile16[i] : tile32[i];
        ka.range = &P.small->ranges[2 * (cls * kBins + i)];
        ka.task_counter = &P.small->counters[counter++];
        const bool alt = cls == 0 && (P.tune.lanes_alt >> tile & 1u);
        const int occ = alt ? P.occ16alt[tile] : cls == 0 ? P.occ16[tile] : P.occ32[tile];
        const int ppt = (cls == 0 ? 2 : 1) * (32 / (alt ? ka_alt_g(tile) : kKaG));
        const int64_t want = (npairs + ppt * (kKaThreads / 32) - 1) / (ppt * (kKaThreads / 32));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)P.nsm * occ));
        const cudaError_t e = alt ? plan_launch_ka_alt(P.mode, tile, ka, grid, stream_for(nlaunch++))
                                  : plan_launch_ka(cls, P.mode, tile, ka, grid, stream_for(nlaunch++));
        if (e != cudaSuccess) return GA_ERR_CUDA;
      }
    }
  }
  {
    KBParams kb{};
    kb.packed_q = P.packed_q;
    kb.packed_t = P.packed_t;
    kb.q_codes = q_codes;
    kb.t_codes = t_codes;
    kb.q_off = q_off;
    kb.t_off = t_off;
    kb.info = P.info;
    kb.sorted = P.sorted;
    kb.range = &P.small->ranges[2 * (kClassLong * kBins)];
    kb.task_counter = &P.small->counters[counter++];
    std::memcpy(kb.tables, P.sc.tables, sizeof(kb.tables));
    std::memcpy(kb.sigma, P.sc.mat, sizeof(kb.sigma));
    kb.A = A;
    kb.alpha = P.sc.alpha;
    kb.beta = P.sc.beta;
    kb.scores = scores;
    kb.bnd = P.bnd;
    kb.bnd_stride = P.bnd_stride;
    const int grid = std::max(P.long_grid, 1);
    const cudaStream_t ls = stream_for(nlaunch++);
    cudaError_t e;
    if (P.long_packed)
      e = P.mode == GA_LOCAL ? launch_kw_local(kb, grid, ls)
        : P.mode == GA_GLOBAL ? launch_kw_global(kb, grid, ls)
                              : launch_kw_semi(kb, grid, ls);
    else if (!dna)
      e = P.mode == GA_LOCAL ? launch_kb_local_prof(kb, grid, P.long_smem, ls)
        : P.mode == GA_GLOBAL ? launch_kb_global_prof(kb, grid, P.long_smem, ls)
                              : launch_kb_semi_prof(kb, grid, P.long_smem, ls);
    else
      e = P.mode == GA_LOCAL ? launch_kb_local_sel(kb, grid, 0, ls)
        : P.mode == GA_GLOBAL ? launch_kb_global_sel(kb, grid, 0, ls)
                              : launch_kb_semi_sel(kb, grid, 0, ls);
    if (e != cudaSuccess) return GA_ERR_CUDA;
  }
  if (conc) {
    for (int i = 0; i < kPlanSide; ++i)
      if (cudaEventRecord(P.join[i], P.side[i]) != cudaSuccess || cudaStreamWaitEvent(s, P.join[i], 0) != cudaSuccess)
        return GA_ERR_CUDA;
  }
  // exact int32 rerun of local int16 pairs that reached the int16 limit
  if (P.mode == GA_LOCAL && dna && n16 > 0) {
    rerun_setup_kernel<<<1, 1, 0, s>>>(P.small->rerun_range, &P.small->rerun_total);
    ka.sorted = P.rerun;
    ka.range = P.small->rerun_range;
    ka.rerun_list = nullptr;
    ka.rerun_count = nullptr;
    ka.task_counter = &P.small->counters[counter++];
    const int tile = kKaNumBins - 1;
    if (plan_launch_ka(1, GA_LOCAL, tile, ka, P.nsm * P.occ32[tile], s) != cudaSuccess) return GA_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

int plan_capture(PlanImpl &P, const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                 const int64_t *t_off, int64_t npairs, int32_t *scores) {
  P.drop_graph();
  cudaStream_t s = P.cap_stream;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GA_ERR_CUDA;
  const int rc = plan_enqueue(P, q_codes, q_off, t_codes, t_off, npairs, scores, s);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || !g) return GA_ERR_CUDA;
  const cudaError_t ei = cudaGraphInstantiate(&P.exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    P.exec = nullptr;
    return GA_ERR_CUDA;
  }
  return GA_OK;
}

int plan_stats(PlanImpl &P, cudaStream_t s, ga_stats *st) {
  Readback *rb = (Readback *)pinned_scratch();
  if (cudaMemcpyAsync(rb, P.small, sizeof(Readback), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GA_ERR_CUDA;
  std::memset(st, 0, sizeof(*st));
  st->cells = (int64_t)rb->cells;
  st->pairs_int32_rerun = rb->rerun_total;
  st->status = rb->status;
  int32_t p16 = 0, p32 = 0, pl = 0;
  for (int b = 0; b < kBins; ++b) {
    p16 += rb->ranges[2 * b + 1] - rb->ranges[2 * b];
    p32 += rb->ranges[2 * (kBins + b) + 1] - rb->ranges[2 * (kBins + b)];
  }
  pl = rb->ranges[2 * (kClassLong * kBins) + 1] - rb->ranges[2 * (kClassLong * kBins)];
  st->pairs_int16 = p16;
  st->pairs_int32 = p32 + pl;
  return GA_OK;
}

// Median device time of `reps` runs (after one untimed run).
int plan_time(PlanImpl &P, const uint8_t *qc, const int64_t *qo, const uint8_t *tc, const int64_t *to,
              int64_t npairs, int32_t *scores, int reps, cudaStream_t s, float *ms) {
  int rc = plan_enqueue(P, qc, qo, tc, to, npairs, scores, s);
  if (rc) return rc;
  std::vector<float> t;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GA_ERR_CUDA;
  for (int r = 0; !rc && r < reps; ++r) {
    cudaEventRecord(e0, s);
    rc = plan_enqueue(P, qc, qo, tc, to, npairs, scores, s);
    cudaEventRecord(e1, s);
    float x = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&x, e0, e1) != cudaSuccess))
      rc = GA_ERR_CUDA;
    t.push_back(x);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return GA_OK;
}

int plan_autotune(PlanImpl &P, const uint8_t *qc, const int64_t *qo, const uint8_t *tc, const int64_t *to,
                  int64_t npairs, int32_t *scores, int reps, cudaStream_t s, ga_tuning *out, float *ms_out) {
  if (reps < 1 || reps > 1000) return GA_ERR_ARG;
  P.drop_graph();
  ga_tuning best = P.tune;
  float tbest = 0.f;
  int rc = plan_time(P, qc, qo, tc, to, npairs, scores, reps, s, &tbest);
  if (rc) return rc;
  auto consider = [&](ga_tuning cand) -> int {
    P.tune = cand;
    float t = 0.f;
    const int r = plan_time(P, qc, qo, tc, to, npairs, scores, reps, s, &t);
    if (r) return r;
    if (t < tbest * 0.99f) {
      tbest = t;
      best = cand;
    }
    P.tune = best;
    return GA_OK;
  };
  // active tiles of the kept tuning that hold pairs of the sample
  auto live_mask = [&](int cls, uint32_t *live) -> int {
    P.tune = best;
    int r = plan_enqueue(P, qc, qo, tc, to, npairs, scores, s);
    if (r) return r;
    Readback *rb = (Readback *)pinned_scratch();
    if (cudaMemcpyAsync(rb, P.small, sizeof(Readback), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return GA_ERR_CUDA;
    const uint32_t mask = cls == 0 ? best.tiles16 : best.tiles32;
    *live = 0;
    for (int b = 0, i = 0; b < kKaNumBins; ++b) {
      if (!(mask >> b & 1u)) continue;
      const int k = cls * kBins + i++;
      if (rb->ranges[2 * k + 1] > rb->ranges[2 * k]) *live |= 1u << b;
    }
    return GA_OK;
  };
  // 1. tiles that no pair of the sample uses: each costs one launch (pairs
  //    of other batches in their range go to the next wider active tile)
  {
    uint32_t l16 = 0, l32 = 0;
    if ((rc = live_mask(0, &l16)) || (rc = live_mask(1, &l32))) return rc;
    if (l16 != best.tiles16 || l32 != best.tiles32) {
      ga_tuning cand = best;
      // keep the widest tile of each class so that the pairs of its range
      // stay on the inter-sequence kernels
      cand.tiles16 = l16 | (best.tiles16 & (1u << (kKaNumBins - 1)));
      cand.tiles32 = l32 | (best.tiles32 & (1u << (kKaNumBins - 1)));
      if (l32 == 0) cand.tiles32 = 0;
      if ((rc = consider(cand))) return rc;
    }
  }
  // 2. bins one after another or concurrent
  {
    ga_tuning cand = best;
    cand.concurrent = !best.concurrent;
    if ((rc = consider(cand))) return rc;
  }
  // 3. greedy removal of non-empty tiles (class by class)
  for (int cls = 0; cls < 2; ++cls) {
    for (;;) {
      uint32_t lm = 0;
      if ((rc = live_mask(cls, &lm))) return rc;
      std::vector<int> live;
      for (int b = 0; b < kKaNumBins; ++b)
        if (lm >> b & 1u) live.push_back(b);
      if (live.size() < 2) break;
      ga_tuning round_best = best;
      float t_round = tbest;
      for (int b : live) {
        ga_tuning cand = best;
        (cls == 0 ? cand.tiles16 : cand.tiles32) &= ~(1u << b);
        P.tune = cand;
        float t = 0.f;
        if ((rc = plan_time(P, qc, qo, tc, to, npairs, scores, reps, s, &t))) return rc;
        if (t < t_round) {
          t_round = t;
          round_best = cand;
        }
      }
      P.tune = best;
      if (t_round < tbest * 0.99f) {
        tbest = t_round;
        best = round_best;
        P.tune = best;
      } else {
        break;
      }
    }
  }
  // 4. alternative lane-group sizes of the live packed tiles: all narrow
  //    tiles with 8 lanes, all wide tiles with 32 lanes, then tile by tile
  //    (one tile alone often moves the whole batch by less than the 1 %
  //    a change must gain)
  {
    uint32_t lm = 0;
    if ((rc = live_mask(0, &lm))) return rc;
    const uint32_t alt = lm & kKaAltTiles;
    uint32_t narrow = 0, wide = 0;
    for (int b = 0; b < kKaNumBins; ++b)
      if (alt >> b & 1u) (ka_alt_g(b) == 8 ? narrow : wide) |= 1u << b;
    for (uint32_t group : {narrow, wide}) {
      if (!group) continue;
      ga_tuning cand = best;
      cand.lanes_alt ^= group;
      if ((rc = consider(cand))) return rc;
    }
    for (int b = 0; b < kKaNumBins; ++b) {
      if (!(alt >> b & 1u)) continue;
      ga_tuning cand = best;
      cand.lanes_alt ^= 1u << b;
      if ((rc = consider(cand))) return rc;
    }
  }
  P.tune = best;
  if (out) *out = best;
  if (ms_out) *ms_out = tbest;
  // leave the sample's scores from the kept tuning
  return plan_enqueue(P, qc, qo, tc, to, npairs, scores, s);
}

}  // namespace
}  // namespace ga

using namespace ga;

extern "C" {

int ga_align_batch(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                   const int64_t *t_off, int64_t npairs, const ga_scoring *scoring, int32_t mode,
                   int32_t *scores, void *stream, ga_stats *stats) {
  return batch_impl(q_codes, q_off, t_codes, t_off, npairs, scoring, mode, scores, stream, stats, 0);
}

static int batch_host_impl(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                           const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                           const int32_t *modes, int32_t nmodes, int32_t *scores, void *stream,
                           ga_stats *stats) {
  if (npairs < 0 || !modes || nmodes < 1 || nmodes > 8) return GA_ERR_ARG;
  for (int k = 0; k < nmodes; ++k)
    if (modes[k] < 0 || modes[k] > 2) return GA_ERR_ARG;
  if (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !scores)) return GA_ERR_ARG;
  {  // the scoring is checked before any stream, copy or allocation is made
    Scoring sc;
    if (int rc0 = check_scoring(scoring, &sc)) return rc0;
  }
  if (npairs == 0) return batch_impl(nullptr, nullptr, nullptr, nullptr, 0, scoring, modes[0], nullptr, stream,
                                     stats, 0);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t qn = q_off[npairs], tn = t_off[npairs];
  if (qn < 0 || tn < 0 || q_off[0] < 0 || t_off[0] < 0 || q_off[0] > qn || t_off[0] > tn) return GA_ERR_ARG;
  // Chunks of pairs: the copies of every chunk go in order on a copy stream,
  // the alignment of chunk k waits only for chunk k's copy, and its scores go
  // back as soon as it is done, so copies and alignment overlap.  Chunk k
  // runs on plan stream k % 2: the readback of its bin populations then waits
  // for chunk k-2 only, so the host enqueues chunk k's kernels while chunk
  // k-1's still run, and the device never drains between chunks.
  const int64_t kChunkPairs = 1 << 18;
  const int nchunk = (int)std::min<int64_t>(8, std::max<int64_t>(1, (npairs + kChunkPairs - 1) / kChunkPairs));
  // geometric chunk sizes (1, 2, 4, ... parts): the first alignment starts
  // after a small copy, and every later copy (host->device bandwidth well
  // above the alignment's input rate) is done before its chunk is reached
  std::vector<int64_t> cut((size_t)nchunk + 1);
  const int64_t parts = ((int64_t)1 << nchunk) - 1;
  for (int k = 0; k <= nchunk; ++k) cut[k] = (int64_t)((double)npairs * (double)(((int64_t)1 << k) - 1) / (double)parts);
  cut[nchunk] = npairs;
  uint8_t *dq = nullptr, *dt = nullptr;
  int64_t *dqo = nullptr, *dto = nullptr;
  int32_t *ds = nullptr;
  cudaStream_t cs = nullptr, pst[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> ev_in((size_t)nchunk, nullptr), ev_done((size_t)nchunk, nullptr);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFreeAsync(dq, s); cudaFreeAsync(dt, s); cudaFreeAsync(dqo, s);
    cudaFreeAsync(dto, s); cudaFreeAsync(ds, s);
  };
  bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&pst[0], cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&pst[1], cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; ok && k < nchunk; ++k)
    ok = cudaEventCreateWithFlags(&ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev_done[k], cudaEventDisableTiming) == cudaSuccess;
  int rc = ok ? GA_OK : GA_ERR_CUDA;
  if (!rc && (pool_malloc((void **)&dq, (size_t)qn + 16, s) != cudaSuccess ||
              pool_malloc((void **)&dt, (size_t)tn + 16, s) != cudaSuccess ||
              pool_malloc((void **)&dqo, sizeof(int64_t) * (size_t)(npairs + 1), s) != cudaSuccess ||
              pool_malloc((void **)&dto, sizeof(int64_t) * (size_t)(npairs + 1), s) != cudaSuccess ||
              pool_malloc((void **)&ds, sizeof(int32_t) * (size_t)(nmodes * npairs + 1), s) != cudaSuccess))
    rc = GA_ERR_OOM;
  cudaEvent_t ready = nullptr;  // the allocations above are ordered on `s`
  if (!rc && (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventRecord(ready, s) != cudaSuccess || cudaStreamWaitEvent(cs, ready, 0) != cudaSuccess ||
              cudaStreamWaitEvent(pst[0], ready, 0) != cudaSuccess ||
              cudaStreamWaitEvent(pst[1], ready, 0) != cudaSuccess))
    rc = GA_ERR_CUDA;
  if (!rc && stats) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  // all copies in, chunk by chunk
  for (int k = 0; !rc && k < nchunk; ++k) {
    const int64_t a = cut[k], b = cut[k + 1];
    const int64_t qa = q_off[a], qb = q_off[b], ta = t_off[a], tb = t_off[b];
    if (qb < qa || tb < ta) {
      rc = GA_ERR_ARG;
      break;
    }
    if (cudaMemcpyAsync(dqo + a, q_off + a, sizeof(int64_t) * (size_t)(b - a + 1), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(dto + a, t_off + a, sizeof(int64_t) * (size_t)(b - a + 1), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        (qb > qa && cudaMemcpyAsync(dq + qa, q_codes + qa, (size_t)(qb - qa), cudaMemcpyHostToDevice, cs) != cudaSuccess) ||
        (tb > ta && cudaMemcpyAsync(dt + ta, t_codes + ta, (size_t)(tb - ta), cudaMemcpyHostToDevice, cs) != cudaSuccess) ||
        cudaEventRecord(ev_in[k], cs) != cudaSuccess)
      rc = GA_ERR_CUDA;
  }
  // align chunk by chunk; scores of a chunk go back behind its alignment
  ga_stats tot{};
  for (int k = 0; !rc && k < nchunk; ++k) {
    const int64_t a = cut[k], b = cut[k + 1];
    cudaStream_t pk = pst[k & 1];
    if (cudaStreamWaitEvent(pk, ev_in[k], 0) != cudaSuccess) {
      rc = GA_ERR_CUDA;
      break;
    }
    KnownRange qr, tr;
    qr.known = tr.known = true;
    qr.start = q_off[a];
    qr.total = q_off[b];
    tr.start = t_off[a];
    tr.total = t_off[b];
    {  // every mode on the chunk copied once (packed once)
      ga_stats st{};
      rc = batch_modes_impl(dq, dqo + a, dt, dto + a, b - a, scoring, modes, nmodes, ds + a, npairs, pk,
                            stats ? &st : nullptr, 0, qr, tr);
      if (!rc && stats) {
        tot.cells += st.cells; tot.pairs += st.pairs; tot.pairs_int16 += st.pairs_int16;
        tot.pairs_int32 += st.pairs_int32; tot.pairs_int32_rerun += st.pairs_int32_rerun;
        tot.dp_ms += st.dp_ms; tot.dp_launches += st.dp_launches; tot.launches += st.launches;
        if (!tot.status) tot.status = st.status;
      }
    }
    if (rc) break;
    if (cudaEventRecord(ev_done[k], pk) != cudaSuccess || cudaStreamWaitEvent(cs, ev_done[k], 0) != cudaSuccess)
      rc = GA_ERR_CUDA;
    for (int md = 0; !rc && md < nmodes; ++md)
      if (cudaMemcpyAsync(scores + (size_t)md * npairs + a, ds + (size_t)md * npairs + a,
                          sizeof(int32_t) * (size_t)(b - a), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        rc = GA_ERR_CUDA;
  }
  // the frees are ordered after the last score copy and everything on the
  // plan streams (also on an error path)
  cudaEvent_t copied = nullptr, tail[2] = {nullptr, nullptr};
  if (cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) == cudaSuccess) {
    cudaEventRecord(copied, cs);
    cudaStreamWaitEvent(s, copied, 0);
  }
  for (int i = 0; i < 2; ++i)
    if (pst[i] && cudaEventCreateWithFlags(&tail[i], cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(tail[i], pst[i]);
      cudaStreamWaitEvent(s, tail[i], 0);
    }
  if (e1) cudaEventRecord(e1, s);
  cleanup();
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = GA_ERR_CUDA;
  if (cs && cudaStreamSynchronize(cs) != cudaSuccess && !rc) rc = GA_ERR_CUDA;
  if (!rc && stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    tot.kernel_ms = ms;
    *stats = tot;
  }
  for (cudaEvent_t e : ev_in) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ev_done) if (e) cudaEventDestroy(e);
  if (ready) cudaEventDestroy(ready);
  if (copied) cudaEventDestroy(copied);
  for (cudaEvent_t e : tail) if (e) cudaEventDestroy(e);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (cs) cudaStreamDestroy(cs);
  for (cudaStream_t p : pst) if (p) cudaStreamDestroy(p);
  return rc;
}

int ga_align_batch_modes(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                         const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                         const int32_t *modes, int32_t nmodes, int32_t *scores, void *stream,
                         ga_stats *stats) {
  return batch_modes_impl(q_codes, q_off, t_codes, t_off, npairs, scoring, modes, nmodes, scores, npairs, stream,
                          stats, 0);
}

int ga_align_batch_host(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                        const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                        int32_t mode, int32_t *scores, void *stream, ga_stats *stats) {
  return batch_host_impl(q_codes, q_off, t_codes, t_off, npairs, scoring, &mode, 1, scores, stream, stats);
}

int ga_align_batch_host_modes(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                              const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                              const int32_t *modes, int32_t nmodes, int32_t *scores, void *stream,
                              ga_stats *stats) {
  return batch_host_impl(q_codes, q_off, t_codes, t_off, npairs, scoring, modes, nmodes, scores, stream, stats);
}

int ga_align_cross(const uint8_t *q_codes, const int64_t *q_off, int64_t nq, const uint8_t *t_codes,
                   const int64_t *t_off, int64_t nt, const ga_scoring *scoring, int32_t mode,
                   int32_t *scores, void *stream, ga_stats *stats) {
  if (nq < 0 || nt < 0 || mode < 0 || mode > 2) return GA_ERR_ARG;
  if (nq > 0 && nt > 0 && (!q_codes || !q_off || !t_codes || !t_off || !scores)) return GA_ERR_ARG;
  Call c((cudaStream_t)stream);
  int rc = check_scoring(scoring, &c.sc);
  if (rc) return rc;
  c.mode = mode;
  c.timing = stats != nullptr;
  Events ev(stats != nullptr, c.s);
  if ((rc = setup(c))) return rc;
  if (nq == 0 || nt == 0) return finish(c, stats, ev.e0, ev.e1, 0);
  if (c.sc.A > 4 && mode == GA_LOCAL)
    return cross_protein_local(c, q_codes, q_off, nq, t_codes, t_off, nt, scores, stats, ev.e0, ev.e1);
  SetView Q{q_codes, q_off, nullptr, nullptr}, T{t_codes, t_off, nullptr, nullptr};
  if ((rc = prepare_set(c, q_codes, q_off, nq, &Q.packed, &Q.bad, &c.small->invalid_q))) return rc;
  if ((rc = prepare_set(c, t_codes, t_off, nt, &T.packed, &T.bad, &c.small->invalid_t))) return rc;
  const int64_t kChunk = 1 << 22;
  const int64_t qpc = std::max<int64_t>(1, std::min<int64_t>(nq, kChunk / nt));
  const int64_t cap = qpc * nt;
  if (cap >= (1ll << 31) - 64) return GA_ERR_ARG;
  uint32_t *keys = c.al.get<uint32_t>((size_t)cap);
  int4 *info = c.al.get<int4>((size_t)cap);
  int32_t *sorted = c.al.get<int32_t>((size_t)cap);
  int32_t *rerun = c.al.get<int32_t>((size_t)cap);
  if (c.al.failed) return GA_ERR_OOM;
  for (int64_t q0 = 0; q0 < nq; q0 += qpc) {
    const int64_t nqc = std::min<int64_t>(qpc, nq - q0);
    rc = run_chunk(c, Q, T, nqc * nt, nt, q0, scores + q0 * nt, 0, keys, info, sorted, rerun);
    if (rc) return rc;
  }
  return finish(c, stats, ev.e0, ev.e1, nq * nt);
}

int ga_align_long(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n, const ga_scoring *scoring,
                  int32_t mode, int32_t *score, void *stream, ga_stats *stats) {
  if (m < 0 || n < 0 || !score || (m > 0 && !q) || (n > 0 && !t)) return GA_ERR_ARG;
  if (mode < 0 || mode > 2) return GA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  {
    Scoring sc;
    const int rc = check_scoring(scoring, &sc);
    if (rc) return rc;
    const int64_t mn = m < n ? m : n;
    if (m >= (1ll << 30) || n >= (1ll << 30) ||
        2 * (int64_t)sc.alpha + (int64_t)sc.beta * (m + n) + 127 * mn >= (1ll << 30))
      return GA_ERR_RANGE;
    // every strip of 512 columns on its own warp, a few rows behind its
    // left neighbour (up to 65536 residues); longer: one warp per pair
    if (m <= 65536 && n <= 65536)
      return sv_align_pair(q, m, t, n, sc.A, sc.mat, sc.alpha, sc.beta, mode, score, s, stats);
  }
  int64_t *off = nullptr;
  if (pool_malloc((void **)&off, 4 * sizeof(int64_t), s) != cudaSuccess) return GA_ERR_OOM;
  fill_off_kernel<<<1, 1, 0, s>>>(off, 0, m);
  fill_off_kernel<<<1, 1, 0, s>>>(off + 2, 0, n);
  const uint8_t *qq = q ? q : (const uint8_t *)off, *tt = t ? t : (const uint8_t *)off;
  int rc = batch_impl(qq, off, tt, off + 2, 1, scoring, mode, score, stream, stats, 1);
  cudaFreeAsync(off, s);
  return rc;
}

int ga_align_banded(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                    const int64_t *t_off, int64_t npairs, const ga_scoring *scoring, const int32_t *w0,
                    int32_t default_w0, int32_t *scores, int32_t *w_used, void *stream, ga_stats *stats) {
  if (npairs < 0 || default_w0 < 0) return GA_ERR_ARG;
  if (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !scores)) return GA_ERR_ARG;
  if (npairs >= (1ll << 31) - 64) return GA_ERR_ARG;
  Call c((cudaStream_t)stream);
  int rc = check_scoring(scoring, &c.sc);
  if (rc) return rc;
  c.mode = GA_GLOBAL;
  if (c.sc.A > 4) {
    // Larger alphabets: exact full DP, no band (w_used = -1).
    rc = batch_impl(q_codes, q_off, t_codes, t_off, npairs, scoring, GA_GLOBAL, scores, stream, stats, 0);
    if (!rc && w_used && npairs > 0) {
      fill_i32_kernel<<<(unsigned)((npairs + 255) / 256), 256, 0, c.s>>>(w_used, npairs, -1);
      if (cudaGetLastError() != cudaSuccess) rc = GA_ERR_CUDA;
    }
    return rc;
  }
  c.timing = stats != nullptr;
  Events ev(stats != nullptr, c.s);
  if ((rc = setup(c))) return rc;
  if (npairs == 0) return finish(c, stats, ev.e0, ev.e1, 0);
  BandRun br(c, q_codes, q_off, t_codes, t_off, npairs);
  if ((rc = br.prepare())) return rc;
  if ((rc = br.plan(w0, default_w0, scores, w_used))) return rc;
  if ((rc = br.launch(w0, default_w0, scores, w_used, nullptr, nullptr))) return rc;
  rc = finish(c, stats, ev.e0, ev.e1, npairs);
  if (!rc && stats) rc = br.band_stats(stats);
  return rc;
}

int ga_band_min_w(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                  const int64_t *t_off, int64_t npairs, const ga_scoring *scoring, int32_t *w_min,
                  int32_t *scores, void *stream, ga_stats *stats) {
  if (npairs < 0) return GA_ERR_ARG;
  if (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !scores || !w_min)) return GA_ERR_ARG;
  if (npairs >= (1ll << 31) - 64) return GA_ERR_ARG;
  Call c((cudaStream_t)stream);
  int rc = check_scoring(scoring, &c.sc);
  if (rc) return rc;
  if (c.sc.A > 4) return GA_ERR_ALPHABET;
  c.mode = GA_GLOBAL;
  c.timing = stats != nullptr;
  Events ev(stats != nullptr, c.s);
  if ((rc = setup(c))) return rc;
  if (npairs == 0) return finish(c, stats, ev.e0, ev.e1, 0);
  BandRun br(c, q_codes, q_off, t_codes, t_off, npairs);
  if ((rc = br.prepare())) return rc;
  int32_t *lo = c.al.get<int32_t>((size_t)npairs), *hi = c.al.get<int32_t>((size_t)npairs);
  if (c.al.failed) return GA_ERR_OOM;
  // doubling from w = 0 brackets the minimal width
  if ((rc = br.plan(nullptr, 0, scores, w_min))) return rc;
  if ((rc = br.launch(nullptr, 0, scores, w_min, nullptr, nullptr))) return rc;
  int32_t *maxgap = &c.small->counters[63];
  const unsigned nb = (unsigned)((npairs + 255) / 256);
  bisect_init_kernel<<<nb, 256, 0, c.s>>>(q_off, t_off, npairs, w_min, lo, hi, maxgap);
  ++c.launches;
  int32_t *h = (int32_t *)pinned_scratch();
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h, maxgap, sizeof(int32_t), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
      cudaStreamSynchronize(c.s) != cudaSuccess)
    return GA_ERR_CUDA;
  int iters = 0;
  while (iters < 31 && ((int64_t)1 << iters) < (int64_t)h[0] + 1) ++iters;
  for (int it = 0; it < iters; ++it)
    if ((rc = br.launch(nullptr, 0, scores, nullptr, lo, hi))) return rc;
  bisect_final_kernel<<<nb, 256, 0, c.s>>>(npairs, lo, w_min);
  ++c.launches;
  if (cudaGetLastError() != cudaSuccess) return GA_ERR_CUDA;
  rc = finish(c, stats, ev.e0, ev.e1, npairs);
  if (!rc && stats) rc = br.band_stats(stats);
  return rc;
}

int ga_band_features(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                     const int64_t *t_off, int64_t npairs, float *features, void *stream,
                     ga_stats *stats) {
  if (npairs < 0 || (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !features)))
    return GA_ERR_ARG;
  return features_impl(q_codes, q_off, t_codes, t_off, npairs, features, nullptr, 0.f, nullptr,
                       nullptr, stream, stats);
}

int ga_band_predict(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                    const int64_t *t_off, int64_t npairs, const uint16_t *params_bf16, float margin,
                    int32_t *w0, float *y, void *stream, ga_stats *stats) {
  if (npairs < 0 ||
      (npairs > 0 && (!q_codes || !q_off || !t_codes || !t_off || !params_bf16 || !w0)))
    return GA_ERR_ARG;
  if (!(margin > -64.f && margin < 64.f)) return GA_ERR_ARG;
  return features_impl(q_codes, q_off, t_codes, t_off, npairs, nullptr, params_bf16, margin, w0, y,
                       stream, stats);
}

const char *ga_strerror(int code) {
  switch (code) {
    case GA_OK: return "ok";
    case GA_ERR_ARG: return "invalid argument";
    case GA_ERR_ALPHABET: return "invalid alphabet or substitution matrix";
    case GA_ERR_OOM: return "device workspace allocation failed";
    case GA_ERR_CUDA: return "CUDA error";
    case GA_ERR_RESIDUE: return "residue code outside the alphabet";
    case GA_ERR_TIMEOUT: return "bounded device wait timed out";
    case GA_ERR_RANGE: return "pair outside the supported range (int32 scores, plan capacity)";
    default: return "unknown error";
  }
}

int ga_version(void) { return 100; }

struct ga_plan {
  ga::PlanImpl *impl;
};

int ga_plan_create(const ga_scoring *scoring, int32_t mode, int64_t max_pairs, int64_t max_residues,
                   int32_t max_len, ga_plan **plan) {
  if (!plan) return GA_ERR_ARG;
  *plan = nullptr;
  ga::PlanImpl *impl = nullptr;
  const int rc = ga::plan_create(scoring, mode, max_pairs, max_residues, max_len, &impl);
  if (rc) return rc;
  *plan = new ga_plan{impl};
  return GA_OK;
}

int ga_plan_run(ga_plan *plan, const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                const int64_t *t_off, int64_t npairs, int32_t *scores, void *stream) {
  if (!plan) return GA_ERR_ARG;
  return ga::plan_enqueue(*plan->impl, q_codes, q_off, t_codes, t_off, npairs, scores, (cudaStream_t)stream);
}

int ga_plan_capture(ga_plan *plan, const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                    const int64_t *t_off, int64_t npairs, int32_t *scores) {
  if (!plan) return GA_ERR_ARG;
  return ga::plan_capture(*plan->impl, q_codes, q_off, t_codes, t_off, npairs, scores);
}

int ga_plan_launch(ga_plan *plan, void *stream) {
  if (!plan || !plan->impl->exec) return GA_ERR_ARG;
  return cudaGraphLaunch(plan->impl->exec, (cudaStream_t)stream) == cudaSuccess ? GA_OK : GA_ERR_CUDA;
}

int ga_plan_stats(ga_plan *plan, void *stream, ga_stats *stats) {
  if (!plan || !stats) return GA_ERR_ARG;
  return ga::plan_stats(*plan->impl, (cudaStream_t)stream, stats);
}

int ga_plan_autotune(ga_plan *plan, const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                     const int64_t *t_off, int64_t npairs, int32_t *scores, int32_t reps, void *stream,
                     ga_tuning *out, float *ms_best) {
  if (!plan) return GA_ERR_ARG;
  return ga::plan_autotune(*plan->impl, q_codes, q_off, t_codes, t_off, npairs, scores, reps,
                           (cudaStream_t)stream, out, ms_best);
}

int ga_plan_get_tuning(const ga_plan *plan, ga_tuning *out) {
  if (!plan || !out) return GA_ERR_ARG;
  *out = plan->impl->tune;
  return GA_OK;
}

int ga_plan_set_tuning(ga_plan *plan, const ga_tuning *tuning) {
  if (!plan || !tuning) return GA_ERR_ARG;
  const uint32_t all = (1u << GA_TILE_COUNT) - 1;
  if ((tuning->tiles16 & ~all) || (tuning->tiles32 & ~all) || tuning->concurrent < 0 || tuning->concurrent > 1 ||
      (tuning->lanes_alt & ~kKaAltTiles))
    return GA_ERR_ARG;
  plan->impl->drop_graph();
  plan->impl->tune = *tuning;
  return GA_OK;
}

int ga_plan_destroy(ga_plan *plan) {
  if (!plan) return GA_ERR_ARG;
  cudaDeviceSynchronize();
  delete plan->impl;
  delete plan;
  return GA_OK;
}

}  // extern "C"
