/*
 * gotoh_plan.h -- batch plans: ga_align_batch with its workspace allocated
 * once, runs that enqueue kernels only (no device allocation, no host
 * synchronisation, so a run can be captured in a CUDA graph and replayed),
 * and an autotuner for the launch configuration of the inter-sequence bins.
 *
 * What a run computes is exactly ga_align_batch (gotoh_align.h): the scores
 * of independent pairs under Eqs. H, E, F of Sec. 2.1 in the plan's mode.
 * The batching is the paper's inter-sequence mapping (Sec. 3.1: many short
 * alignments, one per thread group) with pairs of uneven length sorted into
 * bins of equal tile width; every bin is one persistent kernel launch whose
 * warps pull tasks from a device queue.
 *
 * Life cycle
 *   ga_plan_create   allocates every buffer a run needs for batches of at
 *                    most max_pairs pairs whose residues lie below
 *                    max_residues in each code buffer (q_off[npairs] and
 *                    t_off[npairs] <= max_residues) and whose sequences are
 *                    at most max_len residues long.  It is the only call
 *                    that allocates (cudaMalloc on the current device).
 *   ga_plan_run      enqueues one batch on `stream`: packing, validation,
 *                    planning, the counting sort and every bin kernel, with
 *                    grids fixed by the plan (each kernel reads its bin's
 *                    range from device memory; an empty bin exits at once).
 *                    Safe to call inside stream capture.
 *   ga_plan_capture  records one ga_plan_run for the given pointers and
 *                    npairs into a CUDA graph owned by the plan (replacing
 *                    any earlier one); ga_plan_launch replays it on a
 *                    stream.  A replay reads whatever the captured input
 *                    buffers hold at that time.
 *   ga_plan_stats    synchronises `stream` and reports the last run's
 *                    device status, cell count and int32 reruns.
 *   ga_plan_autotune times candidate tunings on a sample batch and keeps
 *                    the fastest (see ga_tuning); a captured graph is
 *                    dropped when the tuning changes.
 *   ga_plan_destroy  frees everything (synchronises the device first).
 *
 * Arguments of run / capture / autotune: device CSR arrays as for
 * ga_align_batch (q_codes, q_off, t_codes, t_off; int64 offsets,
 * non-decreasing), scores int32[npairs] on the device.  Errors returned at
 * once: GA_ERR_ARG for a null plan or pointer, npairs < 0 or npairs >
 * max_pairs; GA_ERR_CUDA when enqueueing fails.  Errors found on the device
 * (ga_plan_stats().status; affected scores INT32_MIN, all others exact):
 * GA_ERR_RESIDUE, GA_ERR_ARG (decreasing offsets) as for ga_align_batch,
 * and GA_ERR_RANGE for a sequence longer than max_len or ending beyond
 * max_residues (its residues are not read).
 *
 * A plan is used by one host thread at a time; runs of one plan on
 * different streams must not overlap on the GPU (they share the workspace).
 */
#ifndef GOTOH_PLAN_H
#define GOTOH_PLAN_H

#include <stdint.h>

#include "gotoh_align.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Tiles of the inter-sequence kernels: 16 lanes x K columns per pair,
 * K = 6, 7, ..., 20, 24, 32 for tile index 0..16. */
#define GA_TILE_COUNT 17
/* Packed tiles that also exist with another lane-group size of the same
 * width: tiles 0..6 with 8 lanes x 2K columns, tiles 10, 12, 14, 15, 16
 * with 32 lanes x K/2 columns. */
#define GA_TILE_ALT_MASK 0x1d47Fu

/* Launch configuration of a plan.  A set bit k of tiles16 makes tile k a
 * bin of the packed int16x2 kernel: a pair goes to the narrowest active
 * tile at least as wide as its shorter sequence (bin edges = the widths of
 * the active tiles); tiles32 likewise for the int32 kernel.  Pairs wider
 * than every active tile run on the intra-sequence kernel.  A set bit k of
 * lanes_alt (only bits of GA_TILE_ALT_MASK) runs packed tile k with its
 * alternative lane-group size: fewer lanes per pair shorten the wavefront
 * fill of every pair at the cost of more registers per lane, more lanes do
 * the opposite.  concurrent = 1 runs the bins as parallel branches (side
 * streams, graph branches), so that one bin's last tasks overlap the next
 * bin's first; 0 runs them one after another on the caller's stream.
 * Every tuning gives the same (exact) scores; only the time differs. */
typedef struct {
    uint32_t tiles16;
    uint32_t tiles32;
    int32_t concurrent;
    uint32_t lanes_alt;
} ga_tuning;

typedef struct ga_plan ga_plan;

int ga_plan_create(const ga_scoring *scoring, int32_t mode, int64_t max_pairs,
                   int64_t max_residues, int32_t max_len, ga_plan **plan);

int ga_plan_run(ga_plan *plan, const uint8_t *q_codes, const int64_t *q_off,
                const uint8_t *t_codes, const int64_t *t_off, int64_t npairs,
                int32_t *scores, void *stream);

int ga_plan_capture(ga_plan *plan, const uint8_t *q_codes, const int64_t *q_off,
                    const uint8_t *t_codes, const int64_t *t_off, int64_t npairs,
                    int32_t *scores);

/* Replays the captured graph on `stream`; GA_ERR_ARG when nothing has been
 * captured. */
int ga_plan_launch(ga_plan *plan, void *stream);

/* Fills cells, pairs, pairs_int32_rerun and status of the last run or
 * replay; synchronises `stream` (the stream that run was enqueued on). */
int ga_plan_stats(ga_plan *plan, void *stream, ga_stats *stats);

/* Autotuner.  Starting from the current tuning, it times `reps` runs of the
 * sample batch per candidate (median of CUDA-event durations on `stream`)
 * and keeps a candidate only when it saves more than 1 %: first dropping
 * every tile that no pair of the sample uses (one launch each; the widest
 * int16x2 tile stays, and the int32 tiles go when the sample has no int32
 * pair), then bins one after another vs concurrent, then, greedily,
 * removing one active non-empty tile at a time.  Later batches with pairs
 * in a dropped tile's range run on the next wider active tile (or the
 * intra-sequence kernel), so their scores stay exact.
 * The fastest tuning is kept by the plan and copied to *out (nullable);
 * *ms_best (nullable) gets its median time.  `scores` (device,
 * int32[npairs]) receives the sample's scores. */
int ga_plan_autotune(ga_plan *plan, const uint8_t *q_codes, const int64_t *q_off,
                     const uint8_t *t_codes, const int64_t *t_off, int64_t npairs,
                     int32_t *scores, int32_t reps, void *stream, ga_tuning *out,
                     float *ms_best);

int ga_plan_get_tuning(const ga_plan *plan, ga_tuning *out);
/* Sets a tuning (drops a captured graph).  GA_ERR_ARG for bits >= GA_TILE_COUNT
 * or lanes_alt bits outside GA_TILE_ALT_MASK. */
int ga_plan_set_tuning(ga_plan *plan, const ga_tuning *tuning);

int ga_plan_destroy(ga_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* GOTOH_PLAN_H */
