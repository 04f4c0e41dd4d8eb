"""Writes the CPU oracle's scores of two full benchmark workloads to
tests/golden/, so that the GPU tests can compare every output, not a sample:

  long_dna_20k.npz    20,000 long DNA pairs (|Q| ~ U{1000..20000},
                      divergence 1-15 %, indel fraction 10-40 %), global
                      mode, +2/-3, gap open 5, extend 2: 2.8e12 cells;
  serving_200k.npz    the 200,000-request serving stream (60 % DNA +2/-3 5/2,
                      40 % protein BLOSUM62 11/1, 50/50 local/global,
                      lengths LogNormal(median 1000, sigma 1.2) in
                      [100, 50000]).

Every score comes from oracle.batch (the plain int64 recurrence of Sec. 2.1,
Eqs. H, E, F); the inputs come from the seeded generators in synth/.  Each
file also stores a SHA-256 digest of the generated inputs, so a test that
regenerates them can tell a generator change from a wrong score.

    python tests/golden/make_fullsize_goldens.py [--threads N] [long] [serving]

Nothing here imports the CUDA package.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

LONG_PATH = os.path.join(HERE, "long_dna_20k.npz")
SERVING_PATH = os.path.join(HERE, "serving_200k.npz")


def digest(*arrays) -> str:
    """SHA-256 over the raw bytes of the arrays (dtype and shape included)."""
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


def long_digest(b) -> str:
    return digest(b.q_codes, b.q_off, b.t_codes, b.t_off)


def serving_digest(s) -> str:
    return digest(s.q_codes, s.q_off, s.t_codes, s.t_off, s.protein, s.mode)


def make_long(threads: int) -> None:
    b = synth.long_dna_pairs(npairs=20_000)
    t0 = time.time()
    want, errs = oracle.batch(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta,
                              "global", nthreads=threads)
    assert not errs.any()
    np.savez_compressed(LONG_PATH, scores=want.astype(np.int32), digest=np.array(long_digest(b)),
                        cells=np.int64(b.cells()))
    print(f"long: {b.npairs} pairs, {b.cells():.3e} cells, {time.time() - t0:.0f} s", flush=True)


def make_serving(threads: int) -> None:
    s = synth.serving_stream()
    t0 = time.time()
    scores = np.zeros(s.nreq, dtype=np.int64)
    for prot in (False, True):
        for md in (0, 1):
            sel = np.nonzero((s.protein == prot) & (s.mode == md))[0]
            if not len(sel):
                continue
            mat, al, be = s.protein_scoring if prot else s.dna_scoring
            qc, qo = synth.pack_csr([s.q_codes[s.q_off[i]:s.q_off[i + 1]] for i in sel])
            tc, to = synth.pack_csr([s.t_codes[s.t_off[i]:s.t_off[i + 1]] for i in sel])
            want, errs = oracle.batch(qc, qo, tc, to, mat, al, be, "global" if md else "local",
                                      nthreads=threads)
            assert not errs.any()
            scores[sel] = want
    cells = int(np.sum(np.diff(s.q_off) * np.diff(s.t_off)))
    np.savez_compressed(SERVING_PATH, scores=scores.astype(np.int32),
                        digest=np.array(serving_digest(s)), cells=np.int64(cells))
    print(f"serving: {s.nreq} requests, {cells:.3e} cells, {time.time() - t0:.0f} s", flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("which", nargs="*", default=["long", "serving"])
    a = ap.parse_args()
    if "long" in a.which:
        make_long(a.threads)
    if "serving" in a.which:
        make_serving(a.threads)


if __name__ == "__main__":
    main()
