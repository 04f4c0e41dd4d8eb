/*
 * gotoh_oracle.c -- plain CPU oracle for score-only affine-gap (Gotoh)
 * pairwise alignment.  TEST INFRASTRUCTURE ONLY: nothing on the product
 * path (the CUDA library and its Python binding) may link, load or call
 * this file.  Only tests/, the smoke check and the benchmark's CPU
 * baseline leg use it.
 *
 * What it computes (AnySeq/GPU, ICS'22, Sec. 2.1):
 *   H(i,j) = max{ H(i-1,j-1) + sigma(q_i,s_j), E(i,j), F(i,j), nu }   (Eq. H)
 *   E(i,j) = max{ E(i-1,j) - beta,  H(i-1,j) - alpha }               (Eq. E)
 *   F(i,j) = max{ F(i,j-1) - beta,  H(i,j-1) - alpha }               (Eq. F)
 * A gap of length k costs alpha + (k-1)*beta (Sec. 2.1, "Affine Gap
 * Penalty").  Row 0 / column 0 are initialised exactly as the paper's
 * tables for local and global alignment print them; semi-global uses the
 * local tables (Sec. 2.1, "Semi-global Alignments").
 *   local:       nu = 0,    score = max(0, max_{i,j} H(i,j))
 *   global:      nu = -inf, score = H(m,n)
 *   semi-global: nu = -inf, score = max over row m and column n of H,
 *                including H(m,0) and H(0,n).
 * The nu reading for semi-global (-inf, i.e. "free end gaps" / overlap
 * alignment) is a reading of an under-specified sentence; the local-mode
 * nu=0 reading would make semi-global a restricted local alignment.
 *
 * Arithmetic: int64, with -inf represented by GA_ORACLE_NEG = -2^40,
 * far below any reachable score, so -inf minus any number of gap costs
 * can never be confused with a real value.  Three rolling rows: O(n)
 * memory, O(m*n) time, single pass in the paper's row order.
 *
 * Banded global DP (for the band-doubling path): the same recurrence,
 * restricted to cells with lo <= j-i <= hi; every cell outside the band
 * (including row-0 / column-0 initialisation cells) is -inf.  The
 * certificate bound follows the classic band-doubling argument
 * (Ukkonen 1985; Fickett 1984): a global path that visits diagonal d
 * needs at least g(d) = |d| + |d-(n-m)| gap residues, split into at
 * least r(d) runs, so its score is at most
 *     max(sigma_max,0) * (m+n-g)/2 - (alpha*r + beta*(g-r)).
 * This part is not in the paper; it is the reading used for the band
 * certificate.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <stdatomic.h>

#define GA_ORACLE_NEG (-((int64_t)1 << 40))

enum { ORACLE_LOCAL = 0, ORACLE_GLOBAL = 1, ORACLE_SEMIGLOBAL = 2 };

/* flags for oracle_score_ex */
#define ORACLE_FLAG_UNREAD_BORDERS_NEG 1  /* set E(i,0) and F(0,j) to -inf */

static inline int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* status codes written to *err */
#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_RESIDUE 2
#define ORACLE_ERR_OOM 3

/*
 * Full-matrix-semantics score with rolling rows.  Returns the score; on
 * an argument or residue error returns 0 and sets *err.
 * lo/hi restrict the DP to diagonals lo <= j-i <= hi when banded != 0.
 */
/*
 * Region of a banded DP.  block == 0: the band itself, cells with
 * lo <= j-i <= hi (row-0 / column-0 initialisation cells included on the
 * same rule).  block == K > 0: the band rounded out to blocks of K columns
 * (columns bK+1 .. bK+K): for i, j >= 1 the cell is in the region when
 * max(1, bK+1-hi) <= i <= min(m, bK+K-lo); a row-0 cell (0, j) when its
 * block's rows start at 1; a column-0 cell (i, 0) when -i >= lo.  The block
 * region contains the band, so the band certificate (a bound on every path
 * that leaves [lo, hi]) holds for it as well.
 */
static int in_region(int64_t i, int64_t j, int64_t m, int64_t lo, int64_t hi, int64_t block)
{
    if (block <= 0) return (j - i) >= lo && (j - i) <= hi;
    if (j == 0) return -i >= lo;
    int64_t b = (j - 1) / block;
    int64_t r0 = b * block + 1 - hi;
    if (r0 < 1) r0 = 1;
    int64_t r1 = b * block + block - lo;
    if (r1 > m) r1 = m;
    if (i == 0) return r0 == 1;
    return i >= r0 && i <= r1;
}

static int64_t oracle_core(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                           const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                           int32_t mode, int32_t flags, int banded, int64_t lo, int64_t hi,
                           int64_t block, int64_t *Hout, int32_t *err)
{
    *err = ORACLE_OK;
    if (m < 0 || n < 0 || A <= 0 || mode < 0 || mode > 2 || (m > 0 && !q) || (n > 0 && !s) || !sigma) {
        *err = ORACLE_ERR_ARG;
        return 0;
    }
    for (int64_t i = 0; i < m; ++i)
        if (q[i] >= (uint32_t)A) { *err = ORACLE_ERR_RESIDUE; return 0; }
    for (int64_t j = 0; j < n; ++j)
        if (s[j] >= (uint32_t)A) { *err = ORACLE_ERR_RESIDUE; return 0; }

    const int64_t NEG = GA_ORACLE_NEG;
    const int64_t nu = (mode == ORACLE_LOCAL) ? 0 : NEG;
    const int global = (mode == ORACLE_GLOBAL);

    int64_t *Hprev = malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *Hcur = malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *Eprev = malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *Ecur = malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *Fcur = malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!Hprev || !Hcur || !Eprev || !Ecur || !Fcur) {
        free(Hprev); free(Hcur); free(Eprev); free(Ecur); free(Fcur);
        *err = ORACLE_ERR_OOM;
        return 0;
    }

#define IN_BAND(i, j) (!banded || in_region((i), (j), m, lo, hi, block))

    /* Row 0 (paper's initialisation tables). */
    Hprev[0] = IN_BAND(0, 0) ? 0 : NEG;           /* H(0,0) = 0 */
    Eprev[0] = NEG;                               /* E(0,0) = -inf */
    for (int64_t j = 1; j <= n; ++j) {
        int64_t gap = -alpha - beta * (j - 1);
        Hprev[j] = global ? gap : 0;              /* H(0,j) */
        Eprev[j] = NEG;                           /* E(0,j) = -inf */
        if (!IN_BAND(0, j)) Hprev[j] = NEG;
        /* F(0,j) = -alpha - beta*(j-1) in every mode; no later cell reads
         * it (F(i,j) reads F(i,j-1) on the same row i >= 1), so it is not
         * stored here.  ORACLE_FLAG_UNREAD_BORDERS_NEG documents the
         * reading by making no difference. */
    }

    if (Hout) memcpy(Hout, Hprev, (size_t)(n + 1) * sizeof(int64_t));

    int64_t best = 0; /* local: max(0, ...); semi: includes H(m,0), H(0,n) */
    if (mode == ORACLE_SEMIGLOBAL) {
        if (m == 0) {
            for (int64_t j = 0; j <= n; ++j) best = max2(best, Hprev[j]);
        }
        best = max2(best, Hprev[n]); /* H(0,n) */
    }

    for (int64_t i = 1; i <= m; ++i) {
        int64_t col0 = -alpha - beta * (i - 1);
        Hcur[0] = global ? col0 : 0;                                   /* H(i,0) */
        if (!IN_BAND(i, 0)) Hcur[0] = NEG;
        Ecur[0] = (flags & ORACLE_FLAG_UNREAD_BORDERS_NEG) ? NEG : col0; /* E(i,0), never read */
        Fcur[0] = NEG;                                                 /* F(i,0) = -inf */
        const int32_t *srow = sigma + (size_t)q[i - 1] * (size_t)A;
        for (int64_t j = 1; j <= n; ++j) {
            if (!IN_BAND(i, j)) {
                Hcur[j] = NEG; Ecur[j] = NEG; Fcur[j] = NEG;
                continue;
            }
            int64_t e = max2(Eprev[j] - beta, Hprev[j] - alpha);            /* Eq. E */
            int64_t f = max2(Fcur[j - 1] - beta, Hcur[j - 1] - alpha);      /* Eq. F */
            int64_t h = Hprev[j - 1] + (int64_t)srow[s[j - 1]];             /* Eq. H */
            h = max2(h, e);
            h = max2(h, f);
            h = max2(h, nu);
            /* keep -inf cells pinned so that -inf - gaps never drifts */
            if (e < NEG) e = NEG;
            if (f < NEG) f = NEG;
            if (h < NEG) h = NEG;
            Hcur[j] = h; Ecur[j] = e; Fcur[j] = f;
            if (mode == ORACLE_LOCAL) best = max2(best, h);
        }
        if (Hout) memcpy(Hout + (size_t)i * (size_t)(n + 1), Hcur, (size_t)(n + 1) * sizeof(int64_t));
        if (mode == ORACLE_SEMIGLOBAL) {
            best = max2(best, Hcur[n]);                      /* column n */
            if (i == m)
                for (int64_t j = 0; j <= n; ++j) best = max2(best, Hcur[j]); /* row m */
        }
        int64_t *t;
        t = Hprev; Hprev = Hcur; Hcur = t;
        t = Eprev; Eprev = Ecur; Ecur = t;
    }
#undef IN_BAND

    int64_t result;
    if (mode == ORACLE_GLOBAL) result = Hprev[n];
    else result = best;
    free(Hprev); free(Hcur); free(Eprev); free(Ecur); free(Fcur);
    return result;
}

int64_t oracle_score_ex(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                        const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                        int32_t mode, int32_t flags, int32_t *err)
{
    return oracle_core(q, m, s, n, sigma, A, alpha, beta, mode, flags, 0, 0, 0, 0, NULL, err);
}

int64_t oracle_score(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                     const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                     int32_t mode, int32_t *err)
{
    return oracle_core(q, m, s, n, sigma, A, alpha, beta, mode, 0, 0, 0, 0, 0, NULL, err);
}

/* Score plus the full (m+1) x (n+1) H matrix, row-major (small inputs). */
int64_t oracle_matrix(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                      const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                      int32_t mode, int64_t *Hout, int32_t *err)
{
    return oracle_core(q, m, s, n, sigma, A, alpha, beta, mode, 0, 0, 0, 0, 0, Hout, err);
}

/* Global score restricted to diagonals lo <= j-i <= hi (-inf outside). */
int64_t oracle_score_banded(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                            const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                            int64_t lo, int64_t hi, int32_t *err)
{
    return oracle_core(q, m, s, n, sigma, A, alpha, beta, ORACLE_GLOBAL, 0, 1, lo, hi, 0, NULL, err);
}

/* Global score on the band [lo, hi] rounded out to blocks of `block` columns. */
int64_t oracle_score_blockband(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                               const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                               int64_t lo, int64_t hi, int64_t block, int32_t *err)
{
    return oracle_core(q, m, s, n, sigma, A, alpha, beta, ORACLE_GLOBAL, 0, 1, lo, hi, block, NULL,
                       err);
}

/*
 * Upper bound on the score of any global path from (0,0) to (m,n) that
 * visits diagonal d = j - i (band-doubling certificate).
 */
int64_t oracle_band_ub(int64_t m, int64_t n, int64_t sigma_max, int64_t alpha, int64_t beta,
                       int64_t d)
{
    int64_t dn = n - m;
    int64_t lo_main = dn < 0 ? dn : 0, hi_main = dn > 0 ? dn : 0;
    int64_t g = (d < 0 ? -d : d) + ((d - dn) < 0 ? dn - d : d - dn);
    int64_t r = (d < lo_main || d > hi_main) ? 2 : (g > 0 ? 1 : 0);
    int64_t smax = sigma_max > 0 ? sigma_max : 0;
    int64_t diag = (m + n - g) / 2; /* m+n-g is even: g == n-m (mod 2) */
    return smax * diag - (alpha * r + beta * (g - r));
}

/*
 * Band doubling with certificate, global mode.  Starting from w0, the band
 * [min(0,n-m)-w, max(0,n-m)+w] is evaluated; the banded score is accepted
 * when it is >= the bound for the nearest diagonals outside the band, else
 * w doubles (w = max(1, 2w)).  A band that covers the whole matrix is the
 * full DP and is always accepted.  Returns the (exact) score, writes the
 * accepted w, the number of retries and the number of banded cells
 * evaluated over all attempts.
 */
static int64_t doubling_core(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                             const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                             int64_t w0, int64_t block, int64_t *w_used, int64_t *retries,
                             int32_t *err);

int64_t oracle_banded_doubling(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                               const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                               int64_t w0, int64_t *w_used, int64_t *retries, int32_t *err)
{
    return doubling_core(q, m, s, n, sigma, A, alpha, beta, w0, 0, w_used, retries, err);
}

/* Band doubling on block-rounded regions (the GPU's region shape). */
int64_t oracle_banded_doubling_blocks(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                                      const int32_t *sigma, int32_t A, int64_t alpha,
                                      int64_t beta, int64_t w0, int64_t block, int64_t *w_used,
                                      int64_t *retries, int32_t *err)
{
    return doubling_core(q, m, s, n, sigma, A, alpha, beta, w0, block, w_used, retries, err);
}

static int64_t doubling_core(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                             const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                             int64_t w0, int64_t block, int64_t *w_used, int64_t *retries,
                             int32_t *err)
{
    int64_t smax = GA_ORACLE_NEG;
    for (int32_t a = 0; a < A * A; ++a) smax = max2(smax, sigma[a]);
    int64_t dn = n - m;
    int64_t w = w0 < 0 ? 0 : w0;
    int64_t tries = 0;
    for (;;) {
        int64_t lo = (dn < 0 ? dn : 0) - w;
        int64_t hi = (dn > 0 ? dn : 0) + w;
        int64_t sc = oracle_core(q, m, s, n, sigma, A, alpha, beta, ORACLE_GLOBAL, 0, 1, lo, hi,
                                 block, NULL, err);
        if (*err) return 0;
        int covers = (lo <= -m) && (hi >= n);
        int64_t ub = GA_ORACLE_NEG;
        if (lo - 1 >= -m) ub = max2(ub, oracle_band_ub(m, n, smax, alpha, beta, lo - 1));
        if (hi + 1 <= n) ub = max2(ub, oracle_band_ub(m, n, smax, alpha, beta, hi + 1));
        if (covers || sc >= ub) {
            if (w_used) *w_used = w;
            if (retries) *retries = tries;
            return sc;
        }
        w = (w == 0) ? 1 : 2 * w;
        ++tries;
    }
}

/* Smallest w >= 0 whose band (block == 0) or block-rounded band region
 * (block > 0) certifies, by bisection over w.  The certificate is monotone
 * in w: the region only grows with w, so its score can only grow, and the
 * bound of the nearest outside diagonals only shrinks. */
static int64_t min_w_core(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                          const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                          int64_t block, int32_t *err)
{
    int64_t smax = GA_ORACLE_NEG;
    for (int32_t a = 0; a < A * A; ++a) smax = max2(smax, sigma[a]);
    int64_t dn = n - m;
    int64_t lo_w = 0, hi_w = (m > n ? m : n);
    while (lo_w < hi_w) {
        int64_t w = lo_w + (hi_w - lo_w) / 2;
        int64_t lo = (dn < 0 ? dn : 0) - w;
        int64_t hi = (dn > 0 ? dn : 0) + w;
        int64_t sc = oracle_core(q, m, s, n, sigma, A, alpha, beta, ORACLE_GLOBAL, 0, 1, lo, hi,
                                 block, NULL, err);
        if (*err) return -1;
        int covers = (lo <= -m) && (hi >= n);
        int64_t ub = GA_ORACLE_NEG;
        if (lo - 1 >= -m) ub = max2(ub, oracle_band_ub(m, n, smax, alpha, beta, lo - 1));
        if (hi + 1 <= n) ub = max2(ub, oracle_band_ub(m, n, smax, alpha, beta, hi + 1));
        if (covers || sc >= ub) hi_w = w;
        else lo_w = w + 1;
    }
    return lo_w;
}

int64_t oracle_min_certified_w(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                               const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta,
                               int32_t *err)
{
    return min_w_core(q, m, s, n, sigma, A, alpha, beta, 0, err);
}

int64_t oracle_min_certified_w_blocks(const uint8_t *q, int64_t m, const uint8_t *s, int64_t n,
                                      const int32_t *sigma, int32_t A, int64_t alpha,
                                      int64_t beta, int64_t block, int32_t *err)
{
    return min_w_core(q, m, s, n, sigma, A, alpha, beta, block, err);
}

/* ---------------------------------------------------------------------
 * Batch drivers.  One pair per task, tasks handed out through an atomic
 * counter to nthreads POSIX threads (nthreads <= 1: calling thread only).
 * --------------------------------------------------------------------- */
typedef struct {
    const uint8_t *qc; const int64_t *qo; const uint8_t *tc; const int64_t *to;
    int64_t npairs;        /* batch: pairs; cross: nq*nt */
    int64_t nt;            /* cross mode: number of targets, else 0 */
    const int32_t *sigma; int32_t A; int64_t alpha, beta; int32_t mode;
    int64_t *out; int32_t *errs;
    atomic_llong next;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *jb = (batch_job *)arg;
    for (;;) {
        long long p = atomic_fetch_add(&jb->next, 1);
        if (p >= jb->npairs) break;
        int64_t qi = jb->nt ? p / jb->nt : p;
        int64_t ti = jb->nt ? p % jb->nt : p;
        int32_t e = 0;
        int64_t m = jb->qo[qi + 1] - jb->qo[qi];
        int64_t n = jb->to[ti + 1] - jb->to[ti];
        jb->out[p] = oracle_score(jb->qc + jb->qo[qi], m, jb->tc + jb->to[ti], n, jb->sigma,
                                  jb->A, jb->alpha, jb->beta, jb->mode, &e);
        if (jb->errs) jb->errs[p] = e;
    }
    return NULL;
}

static int run_job(batch_job *jb, int32_t nthreads)
{
    atomic_init(&jb->next, 0);
    if (nthreads <= 1) { batch_worker(jb); return 0; }
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return ORACLE_ERR_OOM;
    int32_t started = 0;
    for (int32_t k = 0; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, batch_worker, jb) != 0) break;
        ++started;
    }
    if (started == 0) batch_worker(jb);
    for (int32_t k = 0; k < started; ++k) pthread_join(th[k], NULL);
    free(th);
    return 0;
}

/* scores for pairs p = 0..npairs-1: (q_p, t_p) */
int32_t oracle_batch(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                     const int64_t *t_off, int64_t npairs, const int32_t *sigma, int32_t A,
                     int64_t alpha, int64_t beta, int32_t mode, int64_t *out, int32_t *errs,
                     int32_t nthreads)
{
    batch_job jb = {q_codes, q_off, t_codes, t_off, npairs, 0, sigma, A, alpha, beta, mode,
                    out, errs};
    return run_job(&jb, nthreads);
}

/* scores for all nq x nt (query, target) combinations, row-major [nq][nt] */
int32_t oracle_cross(const uint8_t *q_codes, const int64_t *q_off, int64_t nq,
                     const uint8_t *t_codes, const int64_t *t_off, int64_t nt,
                     const int32_t *sigma, int32_t A, int64_t alpha, int64_t beta, int32_t mode,
                     int64_t *out, int32_t *errs, int32_t nthreads)
{
    if (nt <= 0 || nq <= 0) return 0;
    batch_job jb = {q_codes, q_off, t_codes, t_off, nq * nt, nt, sigma, A, alpha, beta, mode,
                    out, errs};
    return run_job(&jb, nthreads);
}
