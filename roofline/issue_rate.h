/*
 * issue_rate.h -- issue-rate probes behind the integer roofline of the
 * alignment kernels (a measurement library of the benchmark, built as its
 * own libga_roofline.so; the alignment library does not contain it).
 *
 * The DP kernels are bound by integer instruction issue, so their roofline
 * follows the paper's theoretical-peak model (AnySeq/GPU, Sec. 4.2, Eq. TPP
 * and Table 2): cell updates per second <= lanes x clock / ops per cell.
 * rl_issue_rate measures how many lane-operations per second this GPU
 * sustains when nothing but one operation (or one fixed mix of operations)
 * is issued, with 8 independent dependency chains per thread so that the
 * result is a throughput, not a latency.
 *
 *   which    : one of RL_PROBE_* below
 *   iters    : outer iterations; each thread performs iters*16*8 operations
 *              (the mix probes: iters*16*8 packed columns, their ops each)
 *   blocks, threads : launch shape (threads a multiple of 32, <= 1024)
 *   ms       : out, device time of one timed launch (after one warm-up)
 *   lane_ops : out, lane-operations performed by the timed launch
 * Returns 0, 1 (bad argument), 3 (allocation failed) or 4 (CUDA error).
 * The call allocates a 16 KiB sink buffer and synchronises the device.
 */
#ifndef GA_ROOFLINE_ISSUE_RATE_H
#define GA_ROOFLINE_ISSUE_RATE_H

#ifdef __cplusplus
extern "C" {
#endif

#define RL_PROBE_VADD2 0
#define RL_PROBE_VMAXS2 1
#define RL_PROBE_VIADDMAX_S16X2 2
#define RL_PROBE_VIMAX3_S16X2 3
#define RL_PROBE_VIADDMAX_S16X2_RELU 4
#define RL_PROBE_PRMT 5
#define RL_PROBE_IADD 6
#define RL_PROBE_IMAX 7
#define RL_PROBE_VIADDMAX_S32 8
#define RL_PROBE_VIMAX3_S32 9
#define RL_PROBE_IMAD 10
#define RL_PROBE_LOP3 11
#define RL_PROBE_HADD2 12
#define RL_PROBE_HMAX2 13
/* The packed column update of the inter-sequence kernel: prmt (sigma),
 * vadd2 (diagonal + sigma), vimax3 (Eq. H), vadd2 (H - alpha), two
 * viaddmax (Eqs. E and F): 6 ops, 2 cells. */
#define RL_PROBE_MIX_KA 14
/* The same update in int32 cells (one cell): prmt, add, vimax3, add, two
 * viaddmax_s32. */
#define RL_PROBE_MIX_S32 15

int rl_issue_rate(int which, int iters, int blocks, int threads, float *ms, double *lane_ops);

#ifdef __cplusplus
}
#endif

#endif /* GA_ROOFLINE_ISSUE_RATE_H */
