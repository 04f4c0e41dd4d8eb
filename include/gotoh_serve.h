/*
 * gotoh_serve.h -- alignment server: continuous batching of single-pair
 * requests of mixed sizes, alphabets and modes on one GPU.
 *
 * The paper aligns fixed batches (Sec. 4); serving a stream of requests is
 * not in it.  The server keeps one persistent kernel (the strip-task
 * kernel of ga_align_long) fed from a device-resident task queue: every
 * request becomes ceil(max(m, n) / 512) strip tasks, and the strips of one
 * request run on different warps at the same time, so a long request
 * finishes in about the time of its rows rather than of its cells.  A host
 * scheduler thread admits released requests in arrival order while their
 * device memory (codes and strip edges, 8 bytes per row per strip boundary)
 * fits in the arena and a request slot is free, copies them in, appends
 * their tasks and publishes the new queue tail; requests that arrive while
 * others run are admitted as memory and slots free up, and their strips
 * interleave on the device with those already running.  Finished requests
 * leave a completion record (score, status) that the scheduler turns into
 * results with their release / admission / completion times.
 *
 * Scores are those of ga_align_batch for the same pair, mode and scoring
 * (exact int32).  All functions are thread-safe; requests hold host
 * memory only until they are admitted (the server copies them).
 */
#ifndef GOTOH_SERVE_H
#define GOTOH_SERVE_H

#include <stdint.h>

#include "gotoh_align.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GA_SERVE_MAX_LEN 65536   /* longer sequence of a request */
#define GA_SERVE_MAX_SCORINGS 16

typedef struct ga_server ga_server;

typedef struct {
    int64_t arena_bytes;     /* device memory for admitted requests (0: 1 GiB) */
    int32_t max_inflight;    /* request slots (0: 16384) */
    int32_t max_tasks;       /* task ring entries (0: 1 << 20) */
    int32_t device;          /* CUDA device ordinal */
    int32_t idle_us;         /* an idle warp of the persistent kernel exits
                                after this long without work (0: 20000) */
} ga_server_config;

typedef struct {
    int64_t id;              /* as returned by ga_server_submit* */
    int32_t score;           /* INT32_MIN when status != GA_OK */
    int32_t status;          /* GA_OK, GA_ERR_RESIDUE, GA_ERR_TIMEOUT */
    int64_t release_ns;      /* times on the server's clock (ns since creation) */
    int64_t admit_ns;        /* tasks published to the device */
    int64_t done_ns;         /* completion seen by the scheduler */
    int64_t cells;           /* m * n */
} ga_result;

typedef struct {
    int64_t submitted, admitted, completed;
    int64_t cells_completed;
    int64_t arena_high_water;    /* bytes */
    int64_t kernel_launches;     /* launches of the persistent kernel */
    int64_t scheduler_ticks;
    int64_t admit_host_ns;       /* scheduler time: admission decisions and staging */
    int64_t copy_ns;             /* scheduler time: copies in and publication */
    int64_t complete_ns;         /* scheduler time: completion records */
} ga_server_stats;

/* Create a server on cfg->device; *out receives the handle.  GA_ERR_OOM
 * when the device or pinned host memory cannot be allocated. */
int ga_server_create(const ga_server_config *cfg, ga_server **out);

/* Register a scoring scheme (copied); *scoring_id is its index.  Must be
 * called before the requests that use it are submitted. */
int ga_server_add_scoring(ga_server *s, const ga_scoring *scoring, int32_t *scoring_id);

/* Submit npairs requests in CSR form (HOST arrays, copied before return):
 * pair p = query q_codes[q_off[p] .. q_off[p+1]) against target
 * t_codes[t_off[p] .. t_off[p+1]), in mode[p] with scoring_id[p].
 * release_ns (nullable, non-decreasing): the request becomes visible to the
 * scheduler at that time on the server clock (a recorded arrival process);
 * NULL releases them now.  Ids first_id, first_id + 1, ... are assigned in
 * order.  GA_ERR_ARG for a length above GA_SERVE_MAX_LEN, an unknown
 * scoring, a bad mode or decreasing offsets / release times; GA_ERR_OOM for
 * a request that needs more than the whole arena (codes rounded to 16
 * bytes plus 8 * (R + 1) bytes per strip boundary, R = min(m, n)).  On
 * error nothing is submitted. */
int ga_server_submit_batch(ga_server *s, int64_t npairs, const uint8_t *q_codes,
                           const int64_t *q_off, const uint8_t *t_codes, const int64_t *t_off,
                           const int32_t *mode, const int32_t *scoring_id,
                           const int64_t *release_ns, int64_t *first_id);

/* Move up to max finished results into out[]; *count receives how many. */
int ga_server_poll(ga_server *s, ga_result *out, int32_t max, int32_t *count);

/* Wait until every submitted request has completed (or timeout_ms ran out:
 * GA_ERR_TIMEOUT). */
int ga_server_drain(ga_server *s, int64_t timeout_ms);

/* Current time on the server clock (ns since creation). */
int64_t ga_server_clock_ns(ga_server *s);

int ga_server_stats_get(ga_server *s, ga_server_stats *st);

/*
 * ga_probe_bounded_wait -- the strip kernel's bounded wait, run alone: one
 * GPU thread waits (acquire loads, __nanosleep back-off, limit measured on
 * the GPU's globaltimer) until a device flag holding flag_value reaches
 * need.  Nothing writes the flag, so with flag_value < need the wait runs
 * out: *status = GA_ERR_TIMEOUT after about limit_ns; with flag_value >=
 * need, *status = GA_OK at once.  *waited_ns: the time the wait took on the
 * GPU clock.  limit_ns in [0, 1e9], else GA_ERR_ARG; GA_ERR_OOM / GA_ERR_CUDA
 * for allocation or launch failures.  Synchronous (legacy default stream).
 * This is how failure detection of the strip schedule is tested: the wait
 * gives up and reports, and the GPU context stays usable.
 */
int ga_probe_bounded_wait(int32_t flag_value, int32_t need, int64_t limit_ns, int32_t *status,
                          int64_t *waited_ns);

/* Stop the scheduler and the kernel and free everything.  Requests not yet
 * completed are dropped. */
int ga_server_destroy(ga_server *s);

#ifdef __cplusplus
}
#endif

#endif /* GOTOH_SERVE_H */
