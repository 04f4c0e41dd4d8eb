/*
 * gotoh_align.h -- C ABI of libgotoh_gb300.so: score-only affine-gap (Gotoh)
 * pairwise sequence alignment on one GB300 (sm_103a).
 *
 * What is computed (AnySeq/GPU, ICS'22, Sec. 2.1, Eqs. H, E, F):
 *   H(i,j) = max{ H(i-1,j-1) + sigma(q_i,s_j), E(i,j), F(i,j), nu }
 *   E(i,j) = max{ E(i-1,j) - gap_extend, H(i-1,j) - gap_open }
 *   F(i,j) = max{ F(i,j-1) - gap_extend, H(i,j-1) - gap_open }
 * so a gap of k residues costs gap_open + (k-1)*gap_extend (the paper's
 * alpha and beta).  Query residues index rows (i = 1..m), target residues
 * index columns (j = 1..n).  Initialisation and result per mode follow the
 * paper's tables ("Local/Global/Semi-global Alignments"):
 *   GA_LOCAL       nu = 0;    score = max(0, max_{i,j} H(i,j))
 *   GA_GLOBAL      nu = -inf; H(i,0) = -alpha-beta(i-1), H(0,j) likewise;
 *                  score = H(m,n)
 *   GA_SEMIGLOBAL  nu = -inf with the local initialisation (row 0 and
 *                  column 0 are 0); score = max over row m and column n of
 *                  H, including H(m,0) = H(0,n) = 0 (gaps at both ends of
 *                  both sequences are free).
 * Every score is exact (bit-identical to the plain O(mn) recurrence):
 * kernels run packed int16x2 where a static bound or a runtime overflow
 * check proves int16 exact, and int32 otherwise (overflowing int16 pairs
 * are detected and recomputed in int32).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Residues are codes 0..alphabet_size-1 (uint8).  DNA: A,C,G,T = 0..3.
 * Protein: the 24-symbol BLOSUM order ARNDCQEGHILKMFPSTWYVBZX*.
 * Sequences are passed in CSR form: sequence k is codes[off[k] .. off[k+1]).
 *
 * Memory: unless an entry point says "host", every sequence, offset, score
 * and w pointer is a DEVICE pointer owned by the caller (e.g. a torch CUDA
 * tensor).  ga_scoring.matrix is a HOST pointer; it is copied during the
 * call.  The library allocates its own stream-ordered workspace
 * (cudaMallocAsync / cudaFreeAsync on the caller's stream).
 *
 * Execution: work is enqueued asynchronously on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  Scores are valid once the stream has
 * been synchronised.  If `stats` is non-NULL the call synchronises the
 * stream before returning and fills it.  The batch and cross entry points
 * read the bin populations back once per call (a short synchronisation of
 * `stream` between planning and the DP kernels; ga_align_batch_modes plans
 * every mode first and reads all of them back at once) and run the bins as
 * concurrent kernels on four side streams of the library (created once per
 * device, forked from and joined back to `stream` with events).  Calls from
 * different host threads on different streams are safe; their DP kernels
 * may queue behind each other on the shared side streams.  Apart from those
 * streams and the device memory pool the library keeps no global state.
 *
 * Errors returned synchronously (nothing has been enqueued):
 *   GA_ERR_ARG       null pointer where data is required, gap_open <= 0,
 *                    gap_extend <= 0, gap_extend > gap_open, gap costs
 *                    > 4096, a bad mode, negative counts;
 *   GA_ERR_ALPHABET  alphabet_size outside 1..31 or a matrix entry
 *                    outside [-127, 127];
 *   GA_ERR_OOM       workspace allocation failed;
 *   GA_ERR_CUDA      a CUDA call failed while enqueueing.
 * Errors detected on the device (reported through stats->status when
 * stats is non-NULL; the affected scores are set to INT32_MIN, all other
 * scores are exact):
 *   GA_ERR_RESIDUE   a residue code >= alphabet_size;
 *   GA_ERR_ARG       decreasing offsets (negative sequence length);
 *   GA_ERR_RANGE     a pair whose scores could exceed int32
 *                    (|sigma|max * min(m,n) + gap costs >= 2^30);
 *   GA_ERR_TIMEOUT   a bounded device-side wait gave up (never expected;
 *                    reported instead of hanging).
 */
#ifndef GOTOH_ALIGN_H
#define GOTOH_ALIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GA_OK 0
#define GA_ERR_ARG 1
#define GA_ERR_ALPHABET 2
#define GA_ERR_OOM 3
#define GA_ERR_CUDA 4
#define GA_ERR_RESIDUE 5
#define GA_ERR_TIMEOUT 6
#define GA_ERR_RANGE 7

typedef enum { GA_LOCAL = 0, GA_GLOBAL = 1, GA_SEMIGLOBAL = 2 } ga_mode;

/* Substitution matrix and affine gap costs (Sec. 2.1).  matrix is a host
 * pointer to alphabet_size*alphabet_size int8 values, row-major:
 * matrix[a*alphabet_size + b] = sigma(query residue a, target residue b).
 * gap_open = alpha (cost of a gap's first residue), gap_extend = beta
 * (cost of every further residue); 0 < beta <= alpha.  A linear gap
 * penalty is alpha == beta. */
typedef struct {
    int32_t alphabet_size;
    const int8_t *matrix;
    int32_t gap_open;
    int32_t gap_extend;
} ga_scoring;

/* Per-call statistics (filled only when a non-NULL pointer is passed; the
 * call then synchronises its stream). */
typedef struct {
    int64_t cells;             /* sum of m*n over the pairs (full-DP cells) */
    int64_t pairs;             /* pairs (or query x target combinations) */
    int64_t pairs_int16;       /* pairs computed by a packed int16x2 kernel */
    int64_t pairs_int32;       /* pairs routed straight to an int32 kernel */
    int64_t pairs_int32_rerun; /* int16 pairs that overflowed and were redone */
    int64_t band_retries;      /* ga_align_banded: band doublings, all pairs */
    int64_t banded_cells;      /* ga_align_banded: cells evaluated in bands */
    float kernel_ms;           /* device time of the whole call (events) */
    float dp_ms;               /* device time of the DP kernels alone (events
                                  around each DP launch, summed) */
    int32_t dp_launches;       /* DP kernel launches of the call */
    int32_t launches;          /* all kernel launches of the call */
    int32_t status;            /* GA_OK or the first device-detected error */
} ga_stats;

/*
 * ga_align_batch -- independent pairs p = 0..npairs-1: query
 * q_codes[q_off[p] .. q_off[p+1]) against target t_codes[t_off[p] ..
 * t_off[p+1]); scores[p] = the mode's score (Sec. 2.1).  This is the
 * paper's inter-sequence setting (many short alignments, Sec. 3.1 and the
 * all-vs-all read sets of Sec. 4.1).
 *   q_codes, t_codes : device, uint8 residue codes
 *   q_off, t_off     : device, int64[npairs+1], non-decreasing
 *   scores           : device, int32[npairs], written by the call
 * Pairs of any length are accepted: short pairs run on the packed
 * inter-sequence kernels, long ones on the intra-sequence kernel.
 */
int ga_align_batch(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                   const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                   int32_t mode, int32_t *scores, void *stream, ga_stats *stats);

/*
 * ga_align_batch_modes -- ga_align_batch for several modes of the same
 * pairs in one call: both sequence sets are validated and packed once, then
 * each mode in modes[0 .. nmodes) is planned and aligned on the packed
 * copies.
 *   modes  : HOST int32[nmodes], each GA_LOCAL / GA_GLOBAL / GA_SEMIGLOBAL
 *            (repetitions allowed), 1 <= nmodes <= 8
 *   scores : device int32[nmodes * npairs]; scores[k * npairs + p] is pair p
 *            in mode modes[k]
 * Other arguments and errors as for ga_align_batch (GA_ERR_ARG for a bad
 * nmodes or mode); stats (nullable) sums the modes.
 */
int ga_align_batch_modes(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                         const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                         const int32_t *modes, int32_t nmodes, int32_t *scores, void *stream,
                         ga_stats *stats);

/*
 * ga_align_batch_host -- ga_align_batch with every array in HOST memory
 * (pinned memory gives the fastest copies).  The pairs are cut into up to 8
 * chunks of geometrically growing size (one chunk per 2^18 pairs, the
 * first the smallest); all inputs are copied in, chunk by chunk,
 * on a stream of the call's own while the chunks are aligned, each as soon
 * as its inputs have arrived, on two planning streams of the call's own in
 * turn (so that reading back one chunk's bin populations does not wait for
 * the previous chunk's kernels), and its scores copied back behind it;
 * `stream` waits for all of it.  The call synchronises before returning;
 * the host buffers may be reused afterwards.  stats (nullable) sums the chunks' statistics;
 * kernel_ms is the device time of the whole call.
 */
int ga_align_batch_host(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                        const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                        int32_t mode, int32_t *scores, void *stream, ga_stats *stats);

/*
 * ga_align_batch_host_modes -- ga_align_batch_host for several modes of the
 * same pairs: the inputs are copied in once (chunk by chunk, as above) and
 * every mode in modes[0 .. nmodes) runs on each chunk (packed once, as in
 * ga_align_batch_modes), so scoring a batch under, e.g., global and
 * semi-global moves its residues over the host link once instead of once
 * per mode.
 *   modes  : host, int32[nmodes], each GA_LOCAL / GA_GLOBAL / GA_SEMIGLOBAL
 *            (repetitions allowed), 1 <= nmodes <= 8
 *   scores : host, int32[nmodes * npairs]; scores[k * npairs + p] is pair p
 *            in mode modes[k]
 * Errors as for ga_align_batch_host (GA_ERR_ARG for a bad nmodes or mode);
 * stats (nullable) sums all modes and chunks.
 */
int ga_align_batch_host_modes(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                              const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                              const int32_t *modes, int32_t nmodes, int32_t *scores, void *stream,
                              ga_stats *stats);

/*
 * ga_align_cross -- database search: every query k = 0..nq-1 against
 * every target l = 0..nt-1; scores[k*nt + l] (row-major, device,
 * int32[nq*nt]).  Offsets as in ga_align_batch.  The query's scoring
 * profile is staged once in shared memory and the targets stream through
 * it (Sec. 3.1, "scoring profile").  Local searches over alphabets of more
 * than 4 symbols run in packed int16x2; every pair whose int16 running
 * maximum reaches 32767 - sigma_max is recomputed exactly in int32, one
 * pair at a time (a search with many such pairs, e.g. near-identical
 * database hits longer than a few thousand residues, is exact but slow).
 */
int ga_align_cross(const uint8_t *q_codes, const int64_t *q_off, int64_t nq,
                   const uint8_t *t_codes, const int64_t *t_off, int64_t nt,
                   const ga_scoring *scoring, int32_t mode, int32_t *scores, void *stream,
                   ga_stats *stats);

/*
 * ga_align_long -- one long pair (query q[0..m), target t[0..n), device
 * pointers) on the intra-sequence kernel: a thread block whose warps each
 * own a tile of columns and pass boundary cells down the anti-diagonal
 * wavefront (Sec. 3.1, multi-stage partitioning).  *score (device int32)
 * receives the mode's score.
 */
int ga_align_long(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                  const ga_scoring *scoring, int32_t mode, int32_t *score, void *stream,
                  ga_stats *stats);

/*
 * ga_align_banded -- global mode only, exact scores by certified band
 * doubling (not in the paper: the classic Ukkonen/Fickett band bound).
 * For pair p the DP is restricted to diagonals
 *     [min(0,n-m) - w, max(0,n-m) + w]        (d = j - i)
 * starting from w = w0[p] (device int32[npairs]; NULL: default_w0 for all
 * pairs).  The banded score S is accepted when S >= UB, where UB bounds
 * every path that visits the nearest diagonal outside the band:
 *     UB(d) = max(sigma_max,0) * (m+n-g)/2 - (alpha*r + beta*(g-r)),
 *     g = |d| + |d-(n-m)| gap residues in r >= 1 (2 outside the main
 *     diagonals) runs.
 * Otherwise w <- max(1, 2w); a band covering the matrix is the full DP.
 * The kernel evaluates the band rounded out to blocks of 16 target columns
 * (block b = columns 16b+1 .. 16b+16 runs rows max(1, 16b+1-hi) ..
 * min(m, 16b+16-lo)); the rounded region contains the band, so the bound
 * above still certifies it, and it can only accept at a smaller w.
 *   scores : device int32[npairs] -- exact global scores
 *   w_used : device int32[npairs] or NULL -- the accepted w per pair; -1
 *            for pairs that ran as full DP (alphabets of more than 4
 *            symbols, where no banded kernel exists)
 *   w0     : entries < 0 are taken as 0
 * Errors as for ga_align_batch; stats->band_retries and ->banded_cells
 * count doublings and evaluated region cells.
 */
int ga_align_banded(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                    const int64_t *t_off, int64_t npairs, const ga_scoring *scoring,
                    const int32_t *w0, int32_t default_w0, int32_t *scores, int32_t *w_used,
                    void *stream, ga_stats *stats);

/*
 * ga_align_long_noalloc -- ga_align_long for callers that cannot allocate
 * device memory while they align: for example a process whose device memory
 * is held in full by a pooling allocator (cudaMalloc would fail), or a
 * latency-critical loop that cannot take the implicit synchronisation and
 * unbounded latency of cudaMalloc / cudaFree.  The paper has no counterpart;
 * this is a deployment variant of the long-pair kernel.
 *
 * It allocates nothing: its scratch memory (the stage-boundary buffer of the
 * long-pair kernel and a small control block, about 2 MiB) is one
 * file-scope device array that every GPU using the library holds until the
 * process exits.  The caller still passes the inputs q[0..m), t[0..n) and
 * the output *score (all device pointers, as for ga_align_long) and the
 * host scoring struct.
 *   - max(m, n) <= GA_NOALLOC_MAX_LEN, otherwise GA_ERR_ARG (nothing is
 *     enqueued); other argument errors as for ga_align_batch.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) once for that device; make that first call
 *     before any stream capture.  With CUDA's default lazy module loading,
 *     that first call may also be what loads the library's device code and
 *     reserves the array itself (device memory), so make it (a warm-up call
 *     with tiny inputs will do) before a pooling allocator takes the
 *     device's memory, or load modules eagerly (CUDA_MODULE_LOADING=EAGER).
 *     Later calls allocate nothing.
 *   - Every call shares the array and leaves its contents behind; each call
 *     rewrites what must start fresh.  Calls whose GPU work overlaps (other
 *     streams, unordered host threads) race on the array: serialise them.
 *   - A residue code >= alphabet_size yields *score = INT32_MIN.
 */
#define GA_NOALLOC_MAX_LEN 65536
int ga_align_long_noalloc(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n,
                          const ga_scoring *scoring, int32_t mode, int32_t *score, void *stream);

/* Human-readable message for a GA_* code (static string, never NULL). */
const char *ga_strerror(int code);

/* Library ABI version (major*10000 + minor*100 + patch). */
int ga_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GOTOH_ALIGN_H */
