// ga_serve.cu -- host side of the strip-task kernel (ga_serve.cuh):
//   * sv_align_pair: one long pair, all of its strips queued at once, one
//     launch (the multi-warp intra-sequence path of ga_align_long);
//   * the alignment server of include/gotoh_serve.h: a scheduler thread that
//     admits requests by device memory, feeds the device task queue of a
//     persistent ks_kernel and collects completion records.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/gotoh_serve.h"
#include "ga_arena.h"
#include "ga_pool.h"
#include "ga_serve.cuh"
#include "ga_serve_host.h"

namespace ga {

namespace {

cudaError_t sv_prepare_launch(size_t smem, int *blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(ks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, ks_kernel, 32 * kSvWarps, smem);
}

__global__ void sv_oneshot_init_kernel(SvRequest *rq, SvScoring *sc_out, const SvScoring sc,
                                       const uint8_t *q, const uint8_t *t, int2 *edges, int32_t *out,
                                       int m, int n, int mode, int nstrips, int2 *tasks,
                                       unsigned long long *ctr, unsigned long long *cont_seq,
                                       int32_t *stop) {
  const int i = threadIdx.x;
  for (int k = i; k < kSvMaxStrips; k += blockDim.x) {
    rq->progress[k] = 0;
    cont_seq[k] = 0;
  }
  if (i < 8) ctr[i] = 0;
  if (i == 0) {
    tasks[0] = make_int2(0, 0);  // strip 0; the strips after it come as continuations
    *sc_out = sc;
    rq->q = q;
    rq->t = t;
    rq->edges = edges;
    rq->out = out;
    rq->id = 0;
    rq->m = m;
    rq->n = n;
    rq->mode = mode;
    rq->scoring = 0;
    rq->nstrips = nstrips;
    rq->score = (mode == kModeGlobal) ? INT_MIN : 0;
    rq->strips_done = 0;
    rq->status = 0;
    *stop = 1;
  }
  __syncthreads();
  if (i == 0) {
    ctr[1] = 1;  // tail: one task
    ctr[3] = 1;  // one request admitted
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Packed strips keep relative int16 cells exact while sigma_max + alpha <=
// kSvPkMaxStep.
int sv_packed_ok(int A, const int8_t *matrix, int alpha) {
  int smax = 0;
  for (int i = 0; i < A * A; ++i) smax = std::max(smax, (int)matrix[i]);
  return smax + alpha <= kSvPkMaxStep ? 1 : 0;
}

}  // namespace

int sv_strips_for(int64_t m, int64_t n) {
  if (m == 0 || n == 0) return 1;  // closed form, one task
  const int64_t c = m > n ? m : n;
  return (int)std::max<int64_t>(1, (c + kSvW - 1) / kSvW);
}

int sv_align_pair(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n, int A, const int8_t *matrix,
                  int alpha, int beta, int mode, int32_t *score, cudaStream_t s, ga_stats *stats) {
  if (m > kSvMaxLen || n > kSvMaxLen || A < 1 || A > 31) return GA_ERR_ARG;
  SvScoring sc{};
  sc.A = A;
  sc.alpha = alpha;
  sc.beta = beta;
  std::memcpy(sc.sigma, matrix, (size_t)(A * A));
  sc.packed = sv_packed_ok(A, matrix, alpha);
  const int nstrips = sv_strips_for(m, n);
  const int64_t R = m < n ? m : n;
  const size_t o_sc = 0, o_rq = align256(o_sc + sizeof(SvScoring));
  const size_t o_ht = align256(o_rq + sizeof(SvRequest)), o_stop = o_ht + 8 * sizeof(unsigned long long);
  const size_t o_cseq = align256(o_stop + sizeof(int32_t));
  const size_t o_cont = align256(o_cseq + sizeof(unsigned long long) * kSvMaxStrips);
  const size_t o_tasks = align256(o_cont + sizeof(int2) * kSvMaxStrips);
  const size_t o_edges = align256(o_tasks + sizeof(int2));
  const size_t bytes = o_edges + sizeof(int2) * (size_t)(nstrips - 1) * (size_t)(R + 1) + 256;
  char *base = nullptr;
  if (pool_malloc((void **)&base, bytes, s) != cudaSuccess) return GA_ERR_OOM;
  SvScoring *dsc = (SvScoring *)(base + o_sc);
  SvRequest *rq = (SvRequest *)(base + o_rq);
  unsigned long long *ht = (unsigned long long *)(base + o_ht);
  int32_t *stop = (int32_t *)(base + o_stop);
  int2 *tasks = (int2 *)(base + o_tasks);
  int2 *edges = (int2 *)(base + o_edges);
  unsigned long long *cseq = (unsigned long long *)(base + o_cseq);
  int2 *cont = (int2 *)(base + o_cont);

  const size_t smem = (size_t)kSvWarps * (size_t)(sc.A + 1) * kSvW;
  int occ = 0, dev = 0, nsm = 0;
  if (sv_prepare_launch(smem, &occ) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaFreeAsync(base, s);
    return GA_ERR_CUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (stats) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  sv_oneshot_init_kernel<<<1, 128, 0, s>>>(rq, dsc, sc, q, t, edges, score, (int)m, (int)n, mode, nstrips,
                                           tasks, ht, cseq, stop);
  SvParams p{};
  p.req = rq;
  p.scorings = dsc;
  p.tasks = tasks;
  p.task_cap = 1;
  p.head = ht;
  p.tail = ht + 1;
  p.comp = nullptr;
  p.comp_cap = 1;
  p.comp_count = nullptr;
  p.stop = stop;
  p.cont = cont;
  p.cont_seq = cseq;
  p.cont_cap = kSvMaxStrips;
  p.cont_head = ht + 5;
  p.cont_tail = ht + 6;
  p.admitted = ht + 3;
  p.completed = ht + 4;
  p.idle_ns = 0;
  p.wait_ns = 10ll * 1000 * 1000 * 1000;
  p.prof_bytes = (sc.A + 1) * kSvW;
  p.short_chain = 1;  // one pair: each strip warp has a scheduler to itself
  const int grid = std::max(1, std::min((nstrips + kSvWarps - 1) / kSvWarps, nsm * std::max(occ, 1)));
  ks_kernel<<<grid, 32 * kSvWarps, smem, s>>>(p);
  int rc = cudaGetLastError() == cudaSuccess ? GA_OK : GA_ERR_CUDA;
  if (stats && rc == GA_OK) {
    int32_t hst = 0;
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(&hst, &rq->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = GA_ERR_CUDA;
    } else {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      std::memset(stats, 0, sizeof(*stats));
      stats->cells = m * n;
      stats->pairs = 1;
      stats->pairs_int32 = 1;
      stats->kernel_ms = ms;
      stats->dp_ms = ms;
      stats->dp_launches = 1;
      stats->launches = 2;
      stats->status = hst;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(base, s);
  return rc;
}

// ------------------------------------------------------------------------
// The server.
// ------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

// Arena bytes of one admitted request: its codes and its strip edges.
int64_t seq_bytes_for(int64_t m, int64_t n) { return ((((m + 15) & ~15ll) + ((n + 15) & ~15ll)) + 255) & ~255ll; }
int64_t edge_bytes_for(int64_t m, int64_t n) {
  const int64_t R = m < n ? m : n;
  return (int64_t)sizeof(int2) * (sv_strips_for(m, n) - 1) * (R + 1);
}
int64_t request_bytes(int64_t m, int64_t n) {
  return seq_bytes_for(m, n) + ((edge_bytes_for(m, n) + 255) & ~255ll);
}

struct SubmitBatch {
  std::vector<uint8_t> q, t;
  std::vector<int64_t> qo, to;
};

struct Pending {
  std::shared_ptr<SubmitBatch> b;
  int64_t idx;  // pair index in the batch
  int64_t id;
  int32_t mode, scoring;
  int64_t release_ns;
};

struct Inflight {
  bool used = false;
  int64_t id = 0, release_ns = 0, admit_ns = 0, cells = 0;
  int64_t seq_off = -1, seq_bytes = 0;  // codes (in code slab seq_slab)
  int32_t seq_slab = -1;
  int64_t edge_off = -1, edge_bytes = 0;
  int32_t nstrips = 0;
};

}  // namespace

}  // namespace ga

struct ga_server {
  int device = 0;
  ga::Clock::time_point t0;
  int64_t arena_bytes = 0;
  int32_t req_cap = 0;
  int64_t task_cap = 0;
  int64_t idle_ns = 0;
  // device
  uint8_t *arena = nullptr;
  ga::SvRequest *req = nullptr;
  ga::SvScoring *scorings = nullptr;
  int2 *tasks = nullptr;
  unsigned long long *ctr = nullptr;  // head, tail, comp_count, admitted, completed, cont head, cont tail
  int2 *cont = nullptr;               // continuation ring (req_cap entries)
  unsigned long long *cont_seq = nullptr;
  // host (pinned, mapped where the kernel reads or writes it)
  ga::SvCompletion *comp_h = nullptr;
  int32_t *stop_h = nullptr;
  uint8_t *stage_seq = nullptr;
  int64_t stage_seq_cap = 0;
  ga::SvRequest *stage_req = nullptr;
  int2 *stage_tasks = nullptr;
  unsigned long long *stage_tail = nullptr;
  cudaStream_t kstream = nullptr, feed = nullptr;
  bool kernel_running = false;
  bool prev_tick_busy = false;
  size_t smem = 0;
  int grid = 0;
  int max_A = 4;
  // scheduler
  std::thread thr;
  std::mutex mu;
  std::atomic<bool> quit{false};
  std::vector<ga::SvScoring> sc_host;
  std::vector<ga::Pending> pending;   // submitted, FIFO (release order)
  size_t pending_head = 0;
  std::vector<ga_result> done;
  std::vector<ga::Inflight> slots;
  std::unique_ptr<ga::ArenaAlloc> alloc;
  std::unique_ptr<ga::CodeSlabs> slabs;
  int64_t next_id = 0;
  int64_t req_seq = 0;        // requests admitted so far (slot = seq % req_cap)
  unsigned long long tail = 0;
  int64_t tasks_inflight = 0;
  int64_t comp_next = 0;
  int32_t inflight = 0;
  ga_server_stats st{};
  int sched_error = 0;

  int64_t now_ns() const {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(ga::Clock::now() - t0).count();
  }
};

namespace ga {
namespace {

// One scheduler tick: admit, publish, relaunch, collect.  Returns whether
// anything happened.
bool sched_tick(ga_server *S) {
  bool busy = false;
  const int64_t now = S->now_ns();
  int64_t t_a = 0, t_b = 0, t_c = 0;  // phase times of this tick
  // ---- admission decisions (arrival order), under the lock -------------
  struct Adm {
    Pending pd;
    int slot;
    int64_t m, n;
  };
  std::vector<Adm> admit;
  int64_t ntasks = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t stage_bytes = 0;
    while (S->pending_head < S->pending.size()) {
      const Pending &pd = S->pending[S->pending_head];
      if (pd.release_ns > now) break;
      const SubmitBatch &b = *pd.b;
      const int64_t m = b.qo[pd.idx + 1] - b.qo[pd.idx], n = b.to[pd.idx + 1] - b.to[pd.idx];
      const int nstrips = sv_strips_for(m, n);
      const int slot = (int)((S->req_seq + (int64_t)admit.size()) % S->req_cap);
      if (S->slots[slot].used) break;  // slot still busy: keep arrival order
      if (S->tasks_inflight + ntasks + 1 > S->task_cap) break;
      const int64_t seq_bytes = seq_bytes_for(m, n);
      if (stage_bytes + seq_bytes > S->stage_seq_cap) break;
      const int64_t edge_bytes = edge_bytes_for(m, n);
      int64_t eo = -1;
      if (edge_bytes > 0) {
        eo = S->alloc->alloc(edge_bytes);
        if (eo < 0 && S->slabs->trim(*S->alloc)) eo = S->alloc->alloc(edge_bytes);
        if (eo < 0) break;
      }
      int seq_slab = -1;
      const int64_t so = S->slabs->alloc(*S->alloc, seq_bytes, &seq_slab);
      if (so < 0) {
        if (eo >= 0) S->alloc->release(eo, edge_bytes);
        break;
      }
      Inflight &f = S->slots[slot];
      f.used = true;
      f.id = pd.id;
      f.release_ns = pd.release_ns;
      f.cells = m * n;
      f.seq_off = so;
      f.seq_bytes = seq_bytes;
      f.seq_slab = seq_slab;
      f.edge_off = eo;
      f.edge_bytes = edge_bytes;
      f.nstrips = nstrips;
      ntasks += 1;  // strip 0; the kernel queues the others
      stage_bytes += seq_bytes;
      admit.push_back(Adm{pd, slot, m, n});
      ++S->pending_head;
    }
    if (S->pending_head == S->pending.size()) {
      S->pending.clear();
      S->pending_head = 0;
    }
  }
  if (!admit.empty()) {
    // ---- stage codes, records and tasks; copy in and publish (one stream:
    // codes, records, tasks, then the tail) ------------------------------
    int64_t off = 0, k = 0;
    int64_t run_dst = -1, run_src = 0, run_len = 0;  // coalesced code copies
    auto flush_run = [&]() {
      if (run_len > 0)
        cudaMemcpyAsync(S->arena + run_dst, S->stage_seq + run_src, (size_t)run_len,
                        cudaMemcpyHostToDevice, S->feed);
      run_len = 0;
    };
    for (size_t i = 0; i < admit.size(); ++i) {
      const Adm &a = admit[i];
      const Inflight &f = S->slots[a.slot];
      const SubmitBatch &b = *a.pd.b;
      const int64_t mp = (a.m + 15) & ~15ll;
      uint8_t *dst = S->stage_seq + off;
      std::memcpy(dst, b.q.data() + b.qo[a.pd.idx], (size_t)a.m);
      std::memcpy(dst + mp, b.t.data() + b.to[a.pd.idx], (size_t)a.n);
      if (run_len > 0 && run_dst + run_len == f.seq_off && run_src + run_len == off) {
        run_len += f.seq_bytes;
      } else {
        flush_run();
        run_dst = f.seq_off;
        run_src = off;
        run_len = f.seq_bytes;
      }
      SvRequest &r = S->stage_req[i];
      std::memset(&r, 0, sizeof(r));
      r.q = S->arena + f.seq_off;
      r.t = S->arena + f.seq_off + mp;
      r.edges = f.edge_off >= 0 ? (int2 *)(S->arena + f.edge_off) : nullptr;
      r.out = nullptr;
      r.id = a.pd.id;
      r.m = (int32_t)a.m;
      r.n = (int32_t)a.n;
      r.mode = a.pd.mode;
      r.scoring = a.pd.scoring;
      r.nstrips = f.nstrips;
      r.score = a.pd.mode == kModeGlobal ? INT_MIN : 0;
      S->stage_tasks[k] = make_int2(a.slot, 0);
      k += 1;
      off += f.seq_bytes;
    }
    flush_run();
    t_a = S->now_ns();
    const int64_t first_slot = admit[0].slot;
    const int64_t n1 = std::min<int64_t>((int64_t)admit.size(), S->req_cap - first_slot);
    cudaMemcpyAsync(S->req + first_slot, S->stage_req, sizeof(SvRequest) * (size_t)n1,
                    cudaMemcpyHostToDevice, S->feed);
    if ((int64_t)admit.size() > n1)
      cudaMemcpyAsync(S->req, S->stage_req + n1, sizeof(SvRequest) * (admit.size() - n1),
                      cudaMemcpyHostToDevice, S->feed);
    const int64_t t0i = (int64_t)(S->tail % (unsigned long long)S->task_cap);
    const int64_t k1 = std::min<int64_t>(ntasks, S->task_cap - t0i);
    cudaMemcpyAsync(S->tasks + t0i, S->stage_tasks, sizeof(int2) * (size_t)k1, cudaMemcpyHostToDevice,
                    S->feed);
    if (ntasks > k1)
      cudaMemcpyAsync(S->tasks, S->stage_tasks + k1, sizeof(int2) * (size_t)(ntasks - k1),
                      cudaMemcpyHostToDevice, S->feed);
    const unsigned long long new_tail = S->tail + (unsigned long long)ntasks;
    S->stage_tail[0] = new_tail;
    S->stage_tail[1] = (unsigned long long)(S->req_seq + (int64_t)admit.size());  // admitted
    cudaMemcpyAsync(S->ctr + 1, S->stage_tail, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                    S->feed);
    cudaMemcpyAsync(S->ctr + 3, S->stage_tail + 1, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                    S->feed);
    const bool ok = cudaStreamSynchronize(S->feed) == cudaSuccess;
    const int64_t t_admit = S->now_ns();
    t_b = t_admit;
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.admit_host_ns += t_a - now;
    S->st.copy_ns += t_b - t_a;
    if (!ok) S->sched_error = GA_ERR_CUDA;
    S->tail = new_tail;
    for (const Adm &a : admit) S->slots[a.slot].admit_ns = t_admit;
    S->req_seq += (int64_t)admit.size();
    S->tasks_inflight += ntasks;
    S->inflight += (int32_t)admit.size();
    S->st.admitted += (int64_t)admit.size();
    busy = true;
  }
  // ---- keep the persistent kernel running while work is in flight -----
  // The persistent kernel leaves only after idle_ns without work (or at
  // stop): asking the driver whether it is still running costs about as much
  // as admitting a request, so it is asked after an idle tick and every 256
  // ticks, not in every busy tick.
  if (S->kernel_running && (!S->prev_tick_busy || (S->st.scheduler_ticks & 255) == 0) &&
      cudaStreamQuery(S->kstream) == cudaSuccess)
    S->kernel_running = false;
  if (!S->kernel_running && S->inflight > 0) {
    SvParams p{};
    p.req = S->req;
    p.scorings = S->scorings;
    p.tasks = S->tasks;
    p.task_cap = S->task_cap;
    p.head = S->ctr;
    p.tail = S->ctr + 1;
    SvCompletion *comp_d = nullptr;
    int32_t *stop_d = nullptr;
    cudaHostGetDevicePointer((void **)&comp_d, S->comp_h, 0);
    cudaHostGetDevicePointer((void **)&stop_d, S->stop_h, 0);
    p.comp = comp_d;
    p.comp_cap = S->req_cap;
    p.comp_count = S->ctr + 2;
    p.stop = stop_d;
    p.idle_ns = S->idle_ns;
    p.wait_ns = 10ll * 1000 * 1000 * 1000;
    p.prof_bytes = (S->max_A + 1) * kSvW;
    p.cont = S->cont;
    p.cont_seq = S->cont_seq;
    p.cont_cap = S->req_cap;
    p.cont_head = S->ctr + 5;
    p.cont_tail = S->ctr + 6;
    p.admitted = S->ctr + 3;
    p.completed = S->ctr + 4;
    ks_kernel<<<S->grid, 32 * kSvWarps, S->smem, S->kstream>>>(p);
    if (cudaGetLastError() != cudaSuccess) S->sched_error = GA_ERR_CUDA;
    S->kernel_running = true;
    ++S->st.kernel_launches;
    busy = true;
  }
  // ---- completions -----------------------------------------------------
  t_c = S->now_ns();
  int64_t ncomp = 0;
  for (;;) {
    SvCompletion *c = S->comp_h + (S->comp_next % S->req_cap);
    const int64_t seq = *(volatile int64_t *)&c->seq;
    if (seq != S->comp_next + 1) break;
    std::atomic_thread_fence(std::memory_order_acquire);
    const int64_t id = c->id;
    ga_result res{};
    res.id = id;
    res.score = c->score;
    res.status = c->status;
    res.done_ns = S->now_ns();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const int64_t slot = c->slot;
      if (slot >= 0 && slot < S->req_cap && S->slots[slot].used && S->slots[slot].id == id) {
        Inflight &f = S->slots[slot];
        res.release_ns = f.release_ns;
        res.admit_ns = f.admit_ns;
        res.cells = f.cells;
        S->slabs->release(*S->alloc, f.seq_slab);
        if (f.edge_off >= 0) S->alloc->release(f.edge_off, f.edge_bytes);
        S->tasks_inflight -= 1;
        f.used = false;
        --S->inflight;
      } else {
        S->sched_error = GA_ERR_CUDA;  // a record that matches no request
      }
      S->done.push_back(res);
      ++S->st.completed;
      S->st.cells_completed += res.cells;
      S->st.arena_high_water = S->alloc->high_water();
    }
    ++S->comp_next;
    ++ncomp;
    busy = true;
  }
  if (ncomp) {
    const int64_t t_d = S->now_ns();
    std::lock_guard<std::mutex> lk(S->mu);
    S->st.complete_ns += t_d - t_c;
  }
  ++S->st.scheduler_ticks;
  S->prev_tick_busy = busy;
  return busy;
}

void sched_main(ga_server *S) {
  cudaSetDevice(S->device);
  int idle = 0;
  while (!S->quit.load(std::memory_order_acquire)) {
    if (sched_tick(S)) {
      idle = 0;
    } else if (++idle > 64) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

}  // namespace

// One thread waits, with the strip kernel's bounded wait, until *flag >= need.
__global__ void wait_probe_kernel(const int32_t *flag, int32_t need, int64_t limit_ns, int32_t *status,
                                  int64_t *waited_ns) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint64_t t0 = sv_now();
  const bool ok = sv_wait_at_least(flag, need, (uint64_t)limit_ns);
  *waited_ns = (int64_t)(sv_now() - t0);
  *status = ok ? GA_OK : GA_ERR_TIMEOUT;
}

}  // namespace ga

using namespace ga;

extern "C" {

int ga_probe_bounded_wait(int32_t flag_value, int32_t need, int64_t limit_ns, int32_t *status,
                          int64_t *waited_ns) {
  if (!status || !waited_ns || limit_ns < 0 || limit_ns > 1000000000ll) return GA_ERR_ARG;
  struct Buf {
    int32_t flag, status;
    int64_t waited;
  };
  Buf *d = nullptr;
  if (cudaMalloc(&d, sizeof(Buf)) != cudaSuccess) return GA_ERR_OOM;
  Buf h{flag_value, -1, -1};
  int rc = GA_OK;
  if (cudaMemcpy(d, &h, sizeof(Buf), cudaMemcpyHostToDevice) != cudaSuccess) rc = GA_ERR_CUDA;
  if (!rc) {
    wait_probe_kernel<<<1, 32>>>(&d->flag, need, limit_ns, &d->status, &d->waited);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&h, d, sizeof(Buf), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = GA_ERR_CUDA;
  }
  cudaFree(d);
  if (!rc) {
    *status = h.status;
    *waited_ns = h.waited;
  }
  return rc;
}

int ga_server_create(const ga_server_config *cfg, ga_server **out) {
  if (!cfg || !out) return GA_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<ga_server> S(new ga_server());
  S->device = cfg->device;
  S->arena_bytes = cfg->arena_bytes > 0 ? cfg->arena_bytes : (1ll << 30);
  S->req_cap = cfg->max_inflight > 0 ? cfg->max_inflight : 16384;
  S->task_cap = cfg->max_tasks > 0 ? cfg->max_tasks : (1 << 20);
  S->idle_ns = (int64_t)(cfg->idle_us > 0 ? cfg->idle_us : 20000) * 1000;
  if (S->task_cap < kSvMaxStrips) return GA_ERR_ARG;
  if (cudaSetDevice(S->device) != cudaSuccess) return GA_ERR_CUDA;
  S->t0 = Clock::now();
  bool ok = cudaMalloc((void **)&S->arena, (size_t)S->arena_bytes) == cudaSuccess &&
            cudaMalloc((void **)&S->req, sizeof(SvRequest) * (size_t)S->req_cap) == cudaSuccess &&
            cudaMalloc((void **)&S->scorings, sizeof(SvScoring) * GA_SERVE_MAX_SCORINGS) == cudaSuccess &&
            cudaMalloc((void **)&S->tasks, sizeof(int2) * (size_t)S->task_cap) == cudaSuccess &&
            cudaMalloc((void **)&S->ctr, 8 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc((void **)&S->cont, sizeof(int2) * (size_t)S->req_cap) == cudaSuccess &&
            cudaMalloc((void **)&S->cont_seq, sizeof(unsigned long long) * (size_t)S->req_cap) == cudaSuccess &&
            cudaHostAlloc((void **)&S->comp_h, sizeof(SvCompletion) * (size_t)S->req_cap,
                          cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void **)&S->stop_h, 64, cudaHostAllocMapped) == cudaSuccess;
  S->stage_seq_cap = 64ll << 20;
  ok = ok && cudaMallocHost((void **)&S->stage_seq, (size_t)S->stage_seq_cap) == cudaSuccess &&
       cudaMallocHost((void **)&S->stage_req, sizeof(SvRequest) * (size_t)S->req_cap) == cudaSuccess &&
       cudaMallocHost((void **)&S->stage_tasks, sizeof(int2) * (size_t)S->task_cap) == cudaSuccess &&
       cudaMallocHost((void **)&S->stage_tail, 64) == cudaSuccess &&
       cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&S->feed, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    ga_server_destroy(S.release());
    return GA_ERR_OOM;
  }
  std::memset(S->comp_h, 0, sizeof(SvCompletion) * (size_t)S->req_cap);
  *S->stop_h = 0;
  if (cudaMemset(S->ctr, 0, 8 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(S->cont_seq, 0, sizeof(unsigned long long) * (size_t)S->req_cap) != cudaSuccess) {
    ga_server_destroy(S.release());
    return GA_ERR_CUDA;
  }
  S->slots.resize((size_t)S->req_cap);
  S->alloc.reset(new ArenaAlloc(S->arena_bytes));
  S->slabs.reset(new CodeSlabs(S->arena_bytes));
  S->smem = (size_t)kSvWarps * (size_t)(S->max_A + 1) * kSvW;
  int occ = 0, nsm = 0;
  if (sv_prepare_launch(S->smem, &occ) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess) {
    ga_server_destroy(S.release());
    return GA_ERR_CUDA;
  }
  S->grid = nsm * std::max(occ, 1);
  ga_server *raw = S.release();
  raw->thr = std::thread(sched_main, raw);
  *out = raw;
  return GA_OK;
}

int ga_server_add_scoring(ga_server *S, const ga_scoring *sc, int32_t *scoring_id) {
  if (!S || !sc || !scoring_id || !sc->matrix) return GA_ERR_ARG;
  if (sc->alphabet_size < 1 || sc->alphabet_size > 31) return GA_ERR_ALPHABET;
  if (sc->gap_open <= 0 || sc->gap_extend <= 0 || sc->gap_extend > sc->gap_open || sc->gap_open > 4096)
    return GA_ERR_ARG;
  SvScoring h{};
  h.A = sc->alphabet_size;
  h.alpha = sc->gap_open;
  h.beta = sc->gap_extend;
  for (int i = 0; i < h.A * h.A; ++i) {
    if (sc->matrix[i] < -127) return GA_ERR_ALPHABET;
    h.sigma[i] = sc->matrix[i];
  }
  h.packed = sv_packed_ok(h.A, h.sigma, h.alpha);
  std::lock_guard<std::mutex> lk(S->mu);
  if ((int)S->sc_host.size() >= GA_SERVE_MAX_SCORINGS) return GA_ERR_ARG;
  if (S->st.submitted > 0 && h.A > S->max_A) return GA_ERR_ARG;  // profile size is fixed once serving
  const int id = (int)S->sc_host.size();
  S->sc_host.push_back(h);
  if (h.A > S->max_A) {
    S->max_A = h.A;
    S->smem = (size_t)kSvWarps * (size_t)(S->max_A + 1) * kSvW;
    int occ = 0, nsm = 0;
    if (sv_prepare_launch(S->smem, &occ) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess)
      return GA_ERR_CUDA;
    S->grid = nsm * std::max(occ, 1);
  }
  if (cudaMemcpy(S->scorings + id, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return GA_ERR_CUDA;
  *scoring_id = id;
  return GA_OK;
}

int ga_server_submit_batch(ga_server *S, int64_t npairs, const uint8_t *q_codes, const int64_t *q_off,
                           const uint8_t *t_codes, const int64_t *t_off, const int32_t *mode,
                           const int32_t *scoring_id, const int64_t *release_ns, int64_t *first_id) {
  if (!S || npairs < 0 || (npairs > 0 && (!q_off || !t_off || !mode || !scoring_id))) return GA_ERR_ARG;
  if (npairs == 0) return GA_OK;
  const int64_t qn = q_off[npairs] - q_off[0], tn = t_off[npairs] - t_off[0];
  if (qn < 0 || tn < 0 || (qn > 0 && !q_codes) || (tn > 0 && !t_codes)) return GA_ERR_ARG;
  auto b = std::make_shared<SubmitBatch>();
  b->q.assign(q_codes ? q_codes + q_off[0] : nullptr, q_codes ? q_codes + q_off[npairs] : nullptr);
  b->t.assign(t_codes ? t_codes + t_off[0] : nullptr, t_codes ? t_codes + t_off[npairs] : nullptr);
  b->qo.resize((size_t)npairs + 1);
  b->to.resize((size_t)npairs + 1);
  int nsc;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    nsc = (int)S->sc_host.size();
  }
  for (int64_t p = 0; p <= npairs; ++p) {
    b->qo[p] = q_off[p] - q_off[0];
    b->to[p] = t_off[p] - t_off[0];
  }
  for (int64_t p = 0; p < npairs; ++p) {
    const int64_t m = b->qo[p + 1] - b->qo[p], n = b->to[p + 1] - b->to[p];
    if (m < 0 || n < 0 || m > kSvMaxLen || n > kSvMaxLen) return GA_ERR_ARG;
    if (mode[p] < 0 || mode[p] > 2 || scoring_id[p] < 0 || scoring_id[p] >= nsc) return GA_ERR_ARG;
    if (release_ns && p > 0 && release_ns[p] < release_ns[p - 1]) return GA_ERR_ARG;
    if (request_bytes(m, n) > S->arena_bytes) return GA_ERR_OOM;  // could never be admitted
  }
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t now = S->now_ns();
  if (release_ns && !S->pending.empty() && release_ns[0] < S->pending.back().release_ns)
    return GA_ERR_ARG;
  if (first_id) *first_id = S->next_id;
  S->pending.reserve(S->pending.size() + (size_t)npairs);
  for (int64_t p = 0; p < npairs; ++p) {
    Pending pd;
    pd.b = b;
    pd.idx = p;
    pd.id = S->next_id++;
    pd.mode = mode[p];
    pd.scoring = scoring_id[p];
    pd.release_ns = release_ns ? release_ns[p] : now;
    S->pending.push_back(pd);
  }
  S->st.submitted += npairs;
  return GA_OK;
}

int ga_server_poll(ga_server *S, ga_result *out, int32_t max, int32_t *count) {
  if (!S || !count || max < 0 || (max > 0 && !out)) return GA_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const int32_t k = (int32_t)std::min<size_t>((size_t)max, S->done.size());
  std::copy(S->done.begin(), S->done.begin() + k, out);
  S->done.erase(S->done.begin(), S->done.begin() + k);
  *count = k;
  return S->sched_error ? S->sched_error : GA_OK;
}

int ga_server_drain(ga_server *S, int64_t timeout_ms) {
  if (!S) return GA_ERR_ARG;
  const auto end = Clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->sched_error) return S->sched_error;
      if (S->st.completed >= S->st.submitted) return GA_OK;
    }
    if (Clock::now() > end) return GA_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

int64_t ga_server_clock_ns(ga_server *S) { return S ? S->now_ns() : 0; }

int ga_server_stats_get(ga_server *S, ga_server_stats *st) {
  if (!S || !st) return GA_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->st;
  st->arena_high_water = S->alloc ? S->alloc->high_water() : 0;
  return GA_OK;
}

int ga_server_destroy(ga_server *S) {
  if (!S) return GA_ERR_ARG;
  S->quit.store(true, std::memory_order_release);
  if (S->thr.joinable()) S->thr.join();
  cudaSetDevice(S->device);
  if (S->stop_h) *(volatile int32_t *)S->stop_h = 1;
  if (S->kstream) cudaStreamSynchronize(S->kstream);  // warps exit: stop set, bounded idle
  if (S->feed) cudaStreamSynchronize(S->feed);
  cudaFree(S->arena);
  cudaFree(S->req);
  cudaFree(S->scorings);
  cudaFree(S->tasks);
  cudaFree(S->ctr);
  cudaFree(S->cont);
  cudaFree(S->cont_seq);
  cudaFreeHost(S->comp_h);
  cudaFreeHost(S->stop_h);
  cudaFreeHost(S->stage_seq);
  cudaFreeHost(S->stage_req);
  cudaFreeHost(S->stage_tasks);
  cudaFreeHost(S->stage_tail);
  if (S->kstream) cudaStreamDestroy(S->kstream);
  if (S->feed) cudaStreamDestroy(S->feed);
  delete S;
  return GA_OK;
}

}  // extern "C"
