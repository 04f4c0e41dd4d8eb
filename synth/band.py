"""Seeded random draws of the band-predictor training (inputs only).

The network's initial weights and the minibatch order are random numbers
the training draws; they are generated here from explicit seeds and passed
to the training as inputs, so that the CUDA training and the float64 oracle
can start from the same point.  Parameter layout (flat, row-major): W1
64x32, b1 64, W2 64x64, b2 64, w3 64, b3 1 -- 6337 float32 values.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 32, 64
NPARAMS = NH * NIN + NH + NH * NH + NH + NH + 1


def mlp_init(seed: int) -> np.ndarray:
    """He-uniform initial weights, zero biases (float32[NPARAMS])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(NPARAMS, dtype=np.float32)
    k = 0
    p[k:k + NH * NIN] = rng.uniform(-1, 1, size=NH * NIN) * np.sqrt(6.0 / NIN)
    k += NH * NIN + NH
    p[k:k + NH * NH] = rng.uniform(-1, 1, size=NH * NH) * np.sqrt(6.0 / NH)
    k += NH * NH + NH
    p[k:k + NH] = rng.uniform(-1, 1, size=NH) * np.sqrt(3.0 / NH)
    return p


def minibatches(n: int, batch: int, steps: int, seed: int) -> np.ndarray:
    """int32[steps, batch]: epochs of seeded permutations of range(n), cut into batches."""
    rng = np.random.Generator(np.random.PCG64(seed))
    need = steps * batch
    parts, have = [], 0
    while have < need:
        parts.append(rng.permutation(n).astype(np.int32))
        have += n
    return np.concatenate(parts)[:need].reshape(steps, batch)
