"""Learned starting band for banded global alignment (not part of the paper).

Band doubling (``align_banded``) returns exact global scores from any
starting half-width w0; the cost is the cells of every attempt.  Too small a
w0 pays for the failed attempts, too large a w0 for cells outside the
needed band.  This module trains the library's small network to predict a
good w0 per pair and applies it.  Every numerical step runs in the
library's CUDA kernels; this module only sequences the calls:

1. labels: ``band_min_w`` gives each training pair's minimal certified w*
   (the band rounded out to 16-column blocks, as the banded kernel runs it);
2. targets t = log2(1 + w*), features from ``band_features``;
3. ``mlp_train``: Adam on minibatches; the initial weights and the minibatch
   order are inputs (seeded by the caller);
4. margin: the shift of the network output that minimises the banded cells
   of the training pairs, one ``align_banded`` run per candidate;
5. inference: ``band_predict`` (features + network + w0 in one kernel), then
   ``align_banded`` from those w0.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import _binding as B

MARGINS = tuple(np.round(np.arange(-0.5, 1.01, 0.25), 2))
CONSTANT_W0 = (0, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096)


@dataclasses.dataclass
class BandPredictor:
    params_bf16: object        # device int16[6337], bf16 bit patterns
    margin: float = 0.0

    def predict(self, q_codes, q_off, t_codes, t_off, stream=None):
        """(w0, y) per pair, on the device."""
        return B.band_predict(q_codes, q_off, t_codes, t_off, self.params_bf16, self.margin,
                              stream=stream)

    def align(self, q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, stream=None,
              stats: bool = False):
        """Exact global scores by band doubling from the predicted w0."""
        w0, _ = self.predict(q_codes, q_off, t_codes, t_off, stream=stream)
        return B.align_banded(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, w0=w0,
                              stream=stream, stats=stats)


def labels(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, stream=None):
    """(w_min int32[n], scores int32[n]) on the device."""
    return B.band_min_w(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, stream=stream)


def targets_from_w(w_min_host: np.ndarray) -> np.ndarray:
    """t = log2(1 + w*) (float32) for the network's regression."""
    return np.log2(1.0 + np.maximum(np.asarray(w_min_host, dtype=np.float64), 0.0)).astype(np.float32)


def banded_cells(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, w0=None,
                 default_w0: int = 0, stream=None) -> int:
    """Cells evaluated by band doubling from w0 (all attempts)."""
    _, _, st = B.align_banded(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, w0=w0,
                              default_w0=default_w0, stream=stream, stats=True)
    return int(st["banded_cells"])


def best_constant_w0(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend,
                     candidates=CONSTANT_W0, stream=None):
    """(w0, cells) of the constant starting width with the fewest cells."""
    costs = [(banded_cells(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend,
                           default_w0=int(c), stream=stream), int(c)) for c in candidates]
    cells, w0 = min(costs)
    return w0, cells


def train(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, init_params, batch_idx,
          lr: float = 2e-3, margins=MARGINS, w_min=None, stream=None):
    """Train the predictor on the given pairs; returns (BandPredictor, info).

    init_params: float32[6337] initial weights; batch_idx: int32[steps, batch]
    minibatch order (both drawn by the caller); w_min: labels if already known.
    """
    import torch
    dev = q_codes.device
    times = {}

    def mark(name, t0):
        torch.cuda.synchronize(dev)
        times[name] = time.perf_counter() - t0
        return time.perf_counter()
    t0 = time.perf_counter()
    if w_min is None:
        w_min, _ = labels(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend, stream=stream)
    w_host = w_min.cpu().numpy()
    keep = np.nonzero(w_host >= 0)[0]
    feats = B.band_features(q_codes, q_off, t_codes, t_off, stream=stream)
    x = feats[torch.from_numpy(keep).to(dev)].contiguous() if len(keep) < len(w_host) else feats
    t = torch.from_numpy(targets_from_w(w_host[keep])).to(dev)
    bi = np.asarray(batch_idx, dtype=np.int32)
    if len(keep) < len(w_host):  # remap batch indices onto the kept samples
        bi = (bi % len(keep)).astype(np.int32)
    master = torch.from_numpy(np.asarray(init_params, dtype=np.float32).copy()).to(dev)
    wb = B.mlp_cast(master, stream=stream)
    am = torch.zeros_like(master)
    av = torch.zeros_like(master)
    t0 = mark("labels_features", t0)
    losses = B.mlp_train(master, wb, am, av, x, t, torch.from_numpy(bi).to(dev), lr=lr, stream=stream)
    t0 = mark("adam", t0)
    pred = BandPredictor(wb, 0.0)
    costs = []
    for mg in margins:
        pred.margin = float(mg)
        w0, _ = pred.predict(q_codes, q_off, t_codes, t_off, stream=stream)
        costs.append((banded_cells(q_codes, q_off, t_codes, t_off, matrix, gap_open, gap_extend,
                                   w0=w0, stream=stream), float(mg)))
    cells, margin = min(costs)
    pred.margin = margin
    t0 = mark("margin", t0)
    y = B.mlp_forward(wb, x, stream=stream)
    info = {
        "losses": losses.cpu().numpy(),
        "train_pairs": int(len(keep)),
        "margin": margin,
        "train_cells": cells,
        "margin_costs": costs,
        "rmse_log2": float(torch.sqrt(torch.mean((y - t) ** 2)).item()),
        "master": master,
        "seconds": times,
    }
    return pred, info
