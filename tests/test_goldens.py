"""The stored full-size scores (tests/golden/*.npz) are the oracle's.

make_fullsize_goldens.py wrote them from oracle.batch on the seeded inputs
of synth/; here the inputs are generated again, their digest must match the
stored one, and a seeded sample of pairs and requests (the shortest few and
random ones, so that the check takes seconds) is recomputed by the oracle
and compared with the stored scores.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.golden import make_fullsize_goldens as goldens


def _stored(path):
    g = np.load(path)
    return g["scores"].astype(np.int64), str(g["digest"]), int(g["cells"])


def test_long_pair_goldens_are_oracle_scores():
    b = synth.long_dna_pairs(npairs=20_000)
    scores, digest, cells = _stored(goldens.LONG_PATH)
    assert digest == goldens.long_digest(b)
    assert cells == b.cells() and len(scores) == b.npairs
    m, n = b.lengths()
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([np.argsort(m * n)[:6], rng.choice(b.npairs, size=6, replace=False)]))
    sub = b.subset(idx)
    want, errs = oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, b.matrix, b.alpha, b.beta,
                              "global", nthreads=4)
    assert not errs.any()
    np.testing.assert_array_equal(scores[idx], want)


def test_serving_goldens_are_oracle_scores():
    s = synth.serving_stream()
    scores, digest, cells = _stored(goldens.SERVING_PATH)
    assert digest == goldens.serving_digest(s)
    assert len(scores) == s.nreq
    assert cells == int(np.sum(np.diff(s.q_off) * np.diff(s.t_off)))
    rng = np.random.default_rng(12)
    size = np.diff(s.q_off) * np.diff(s.t_off)
    small = np.nonzero(size < 400_000)[0]
    idx = rng.choice(small, size=40, replace=False)
    for i in idx:
        mat, al, be = s.protein_scoring if s.protein[i] else s.dna_scoring
        q = s.q_codes[s.q_off[i]:s.q_off[i + 1]]
        t = s.t_codes[s.t_off[i]:s.t_off[i + 1]]
        assert scores[i] == oracle.score(q, t, mat, al, be, "global" if s.mode[i] else "local"), i
