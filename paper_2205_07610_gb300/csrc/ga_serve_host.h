// ga_serve_host.h -- entry of the strip-task pipeline for one pair, called
// by ga_align_long (plain types only, so that the kernel is compiled in one
// translation unit).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gotoh_align.h"

namespace ga {

// Score of one pair (device codes q[0..m), t[0..n)) with every strip of
// 512 columns of the longer sequence on its own warp.  The scoring has
// been validated by the caller.  GA_ERR_ARG when max(m, n) > 65536.
int sv_align_pair(const uint8_t *q, int64_t m, const uint8_t *t, int64_t n, int A, const int8_t *matrix,
                  int alpha, int beta, int mode, int32_t *score, cudaStream_t s, ga_stats *stats);

int sv_strips_for(int64_t m, int64_t n);

}  // namespace ga
