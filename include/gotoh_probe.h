/*
 * gotoh_probe.h -- issue-rate probes for the integer roofline.
 *
 * The DP kernels are bound by integer instruction issue, so their roofline
 * follows the paper's theoretical-peak model (AnySeq/GPU, Sec. 4.2, Eq. TPP
 * and Table 2): cell updates per second <= #lanes x clock / ops-per-cell.
 * ga_probe_issue_rate measures, for one operation of the cell update, how
 * many lane-operations per second this GPU sustains when nothing but that
 * operation is issued (8 independent dependency chains per thread, so the
 * result is a throughput, not a latency).
 *
 *   which    : one of GA_PROBE_* below
 *   iters    : outer iterations; each thread performs iters*16*8 operations
 *              (GA_PROBE_CELL: iters*16*8 packed columns of 6 ops each)
 *   blocks, threads : launch shape (threads a multiple of 32, <= 1024)
 *   ms       : out, device time of one timed launch (after one warm-up)
 *   lane_ops : out, lane-operations performed by the timed launch
 * Returns 0, 1 (bad argument), 3 (allocation failed) or 4 (CUDA error).
 * The call allocates a 16 KiB sink buffer and synchronises the device.
 */
#ifndef GOTOH_PROBE_H
#define GOTOH_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

#define GA_PROBE_VADD2 0
#define GA_PROBE_VMAXS2 1
#define GA_PROBE_VIADDMAX_S16X2 2
#define GA_PROBE_VIMAX3_S16X2 3
#define GA_PROBE_VIADDMAX_S16X2_RELU 4
#define GA_PROBE_PRMT 5
#define GA_PROBE_IADD 6
#define GA_PROBE_IMAX 7
#define GA_PROBE_VIADDMAX_S32 8
#define GA_PROBE_VIMAX3_S32 9
#define GA_PROBE_IMAD 10
#define GA_PROBE_LOP3 11
#define GA_PROBE_HADD2 12
#define GA_PROBE_HMAX2 13
#define GA_PROBE_CELL 14

int ga_probe_issue_rate(int which, int iters, int blocks, int threads, float *ms,
                        double *lane_ops);

#ifdef __cplusplus
}
#endif

#endif /* GOTOH_PROBE_H */
