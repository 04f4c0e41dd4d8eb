"""GB300-native score-only affine-gap (Gotoh) pairwise alignment.

The hot path is the CUDA library ``_lib/libgotoh_gb300.so`` (C ABI in
``include/gotoh_align.h``, sm_103a kernels in ``csrc/``); this package is a
thin ctypes binding with the same entry points.  Modes follow Sec. 2.1 of the
AnySeq/GPU paper: local (Smith-Waterman), global (Needleman-Wunsch) and
semi-global, with a substitution matrix and affine gaps (gap of k residues
costs gap_open + (k-1) * gap_extend).
"""
from ._binding import (LOCAL, GLOBAL, SEMIGLOBAL, EXPORTED, GotohError, Scoring, Stats,
                       align_banded, align_batch, align_batch_modes, align_batch_host, align_batch_host_modes,
                       align_cross,
                       align_long,
                       align_long_noalloc, NOALLOC_MAX_LEN, probe_bounded_wait,
                       lib_path, load, make_scoring, strerror, version, BAND_NFEAT, MLP_NPARAMS,
                       band_features, band_min_w, band_predict, mlp_forward, mlp_loss_grad,
                       mlp_train, mlp_cast, Server, RESULT_DTYPE, SERVE_MAX_LEN, Plan, Tuning,
                       TILE_K, TILE_ALT_MASK)
from .build import build

__all__ = [
    "LOCAL", "GLOBAL", "SEMIGLOBAL", "EXPORTED", "GotohError", "Scoring", "Stats", "align_banded",
    "align_batch", "align_batch_modes", "align_batch_host", "align_batch_host_modes", "align_cross", "align_long", "align_long_noalloc",
    "NOALLOC_MAX_LEN", "probe_bounded_wait", "lib_path", "load",
    "make_scoring", "strerror", "version", "build", "BAND_NFEAT", "MLP_NPARAMS", "band_features",
    "band_min_w", "band_predict", "mlp_forward", "mlp_loss_grad", "mlp_train", "mlp_cast",
    "Server", "RESULT_DTYPE", "SERVE_MAX_LEN", "Plan", "Tuning", "TILE_K", "TILE_ALT_MASK",
]
