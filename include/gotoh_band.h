/*
 * gotoh_band.h -- C ABI of the learned band predictor for banded global
 * alignment (ga_align_banded in gotoh_align.h).
 *
 * None of this is in the AnySeq/GPU paper.  Banded global alignment with
 * band doubling (the Ukkonen/Fickett bound) is exact whatever band it starts
 * from; a good starting half-width w0 saves the doublings (too narrow) and
 * the wasted cells (too wide).  The predictor is a small network over cheap
 * pair features, trained on the minimal certified widths that the library
 * itself computes (ga_band_min_w).
 *
 * Conventions as in gotoh_align.h: every array is a DEVICE pointer owned by
 * the caller (sequences as uint8 codes + int64 CSR offsets), calls enqueue
 * on `stream` (NULL = legacy default stream) unless stated otherwise,
 * return a GA_* code synchronously, and report device-detected errors
 * (GA_ERR_RESIDUE, ...) through stats->status.  All entry points here are
 * for DNA (codes 0..3); a code >= 4 is GA_ERR_RESIDUE.
 */
#ifndef GOTOH_BAND_H
#define GOTOH_BAND_H

#include <stdint.h>

#include "gotoh_align.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GA_BAND_NFEAT 32
#define GA_MLP_HIDDEN 64
/* W1[64][32], b1[64], W2[64][64], b2[64], w3[64], b3 -- row-major, in this
 * order, as float32 (master) or bf16 bit patterns (uint16). */
#define GA_MLP_NPARAMS 6337

/*
 * ga_band_features -- the 32 features of each pair p, written to
 * features[p*32 .. p*32+31] (device float32[npairs*32]).  With k-mers of 12
 * residues, the k-mers of Q at positions 0, s, 2s, ... (s = max(1,
 * ceil((m-11)/2048)), at most 2048 samples) are matched against every
 * k-mer of S; a hit (i, j) has diagonal d = j - i and excursion
 * e = d - clamp(d, min(0,n-m), max(0,n-m)).  Features: log2(1+m)/16,
 * log2(1+n)/16, log2(1+|n-m|)/16, min(m,n)/max(m,n), matched samples /
 * samples, log2(1+hits)/16, per eighth of Q matched / samples (8), the
 * histogram of min(15, bitlength|e|) over hits (16), the fraction of hits
 * with e < 0, and 1/s.  Quotients with a zero denominator are 0.
 */
int ga_band_features(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                     const int64_t *t_off, int64_t npairs, float *features, void *stream,
                     ga_stats *stats);

/*
 * ga_band_min_w -- for each global pair, the smallest w >= 0 whose band
 * (rounded out to 16-column blocks, as ga_align_banded evaluates it) is
 * certified, i.e. the training label of the predictor; scores[p] receives
 * the exact global score.  Band doubling from w = 0 brackets w_min in
 * (w/2, w]; bisection steps over all pairs at once then narrow every
 * bracket to one value (certification is monotone in w).  Invalid pairs get
 * w_min = -1.  Synchronises the stream (it reads back the bracket widths).
 */
int ga_band_min_w(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                  const int64_t *t_off, int64_t npairs, const ga_scoring *scoring, int32_t *w_min,
                  int32_t *scores, void *stream, ga_stats *stats);

/*
 * ga_band_predict -- features and network fused in one kernel: per pair
 * y = net(features) (written to y[p] when y != NULL) and the starting band
 *     w0[p] = clamp(ceil(2^clamp(y + margin, 0, 30)) - 1, 0, min(m, n)),
 * ready to pass to ga_align_banded.  params_bf16: device uint16[6337].
 */
int ga_band_predict(const uint8_t *q_codes, const int64_t *q_off, const uint8_t *t_codes,
                    const int64_t *t_off, int64_t npairs, const uint16_t *params_bf16, float margin,
                    int32_t *w0, float *y, void *stream, ga_stats *stats);

/*
 * ga_mlp_forward -- y[b] = net(x[b*32 .. b*32+31]) for b < n, float32
 * arithmetic with the bf16 weights params_bf16 (device uint16[6337]):
 *     h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3,
 * every dot product accumulated in index order with fused multiply-adds.
 */
int ga_mlp_forward(const uint16_t *params_bf16, const float *x, int64_t n, float *y, void *stream);

/*
 * ga_mlp_loss_grad -- loss L = sum_b (y_b - t_b)^2 / (2n) over the n
 * samples (x: float32[n*32], target: float32[n]) and its gradient with
 * respect to the bf16 weights, grad: float32[6337] (same layout), loss:
 * float32[1] or NULL.  Batch sums run in sample order (deterministic).
 */
int ga_mlp_loss_grad(const uint16_t *params_bf16, const float *x, const float *target, int32_t n,
                     float *grad, float *loss, void *stream);

/*
 * ga_mlp_train -- `steps` Adam steps (Kingma & Ba) on minibatches
 * batch_idx[k*batch .. (k+1)*batch) (device int32, each in [0, nsamples))
 * of the samples (x, target).  Each step takes the forward/backward pass
 * with the bf16 copy, updates the float32 master weights and the moments
 * adam_m, adam_v (device float32[6337] each, zero before the first step),
 * and refreshes params_bf16 (round to nearest even).  Bias correction
 * uses step numbers step0+1 .. step0+steps.  losses: device
 * float32[steps] or NULL, the loss of each minibatch.  The steps run as one
 * CUDA graph when `stream` is a created stream not being captured.
 * Synchronises the stream; GA_ERR_ARG also when a batch index is out of
 * range.
 */
int ga_mlp_train(float *master, uint16_t *params_bf16, float *adam_m, float *adam_v, const float *x,
                 const float *target, int64_t nsamples, const int32_t *batch_idx, int32_t steps,
                 int32_t batch, int32_t step0, float lr, float beta1, float beta2, float eps,
                 float *losses, void *stream);

/* ga_mlp_cast -- params_bf16 = bf16(master), round to nearest even. */
int ga_mlp_cast(const float *master, uint16_t *params_bf16, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GOTOH_BAND_H */
