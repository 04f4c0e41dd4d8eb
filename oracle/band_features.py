"""Pair features of the band predictor -- TEST INFRASTRUCTURE (oracle).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use this module.  The product computes the same features in its own CUDA
kernel; the two share no code.

The band predictor is not part of the paper.  It estimates, for a global
pair, the smallest band half-width w whose certified band-doubling attempt
succeeds (the Ukkonen/Fickett band bound), from cheap sequence statistics:
lengths, a k-mer sketch similarity and a histogram of the diagonals on which
the two sequences share k-mers.  This file is the definition of those
statistics, written out plainly with numpy (no hashing, no blocking).

Definition, for DNA codes (0..3) Q of length m and S of length n:

* k-mers: KMER = 12 consecutive codes read as a base-4 number, first code
  most significant; Q has nq = max(0, m - KMER + 1) of them, S has
  max(0, n - KMER + 1).
* Sketch of Q: the k-mers at positions i = 0, s, 2s, ... < nq with stride
  s = max(1, ceil(nq / MAX_SAMPLES)); ns of them.  Every k-mer of S is used.
* Hits: every pair (i, j), i a sampled position of Q and j any position of
  S, whose k-mers are equal.  H = number of hits.  The hit's diagonal is
  d = j - i and its excursion e = d - clamp(d, min(0, n-m), max(0, n-m))
  (the distance by which it leaves the strip of main diagonals).
* A sampled position is matched when it is in at least one hit.  Segment of
  position i: seg = (NSEG * i) // nq.

Features (float32; log2 terms computed in float32, every other one an exact
IEEE float32 quotient of integers):
  0  log2(1 + m) / 16            1  log2(1 + n) / 16
  2  log2(1 + |n - m|) / 16      3  min(m, n) / max(m, n)
  4  matched / ns                5  log2(1 + H) / 16
  6..13   per segment: matched in segment / sampled in segment
  14..29  per bin b: hits with bin(|e|) = b, over H;  bin(a) = min(15, bitlength(a))
  30  hits with e < 0, over H    31  1 / s
Quotients with a zero denominator are 0.
"""
from __future__ import annotations

import numpy as np

KMER = 12
MAX_SAMPLES = 2048
NSEG = 8
NBINS = 16
NFEAT = 32


def kmers(codes: np.ndarray) -> np.ndarray:
    """All k-mers of a code array as int64 base-4 numbers (first code most significant)."""
    codes = np.asarray(codes, dtype=np.int64)
    nk = len(codes) - KMER + 1
    if nk <= 0:
        return np.zeros(0, dtype=np.int64)
    v = np.zeros(nk, dtype=np.int64)
    for u in range(KMER):
        v = (v << 2) | codes[u:u + nk]
    return v


def sample_stride(m: int) -> int:
    nq = max(0, m - KMER + 1)
    return max(1, -(-nq // MAX_SAMPLES)) if nq > 0 else 1


def hits(q: np.ndarray, s: np.ndarray):
    """(i, j) arrays of every hit, sampled positions and the stride."""
    m = len(q)
    nq = max(0, m - KMER + 1)
    stride = sample_stride(m)
    qi = np.arange(0, nq, stride, dtype=np.int64)
    qk = kmers(q)[qi] if nq > 0 else np.zeros(0, dtype=np.int64)
    sk = kmers(s)
    if len(qi) == 0 or len(sk) == 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z, qi, stride
    order = np.argsort(qk, kind="stable")
    qsorted, qpos = qk[order], qi[order]
    lo = np.searchsorted(qsorted, sk, "left")
    hi = np.searchsorted(qsorted, sk, "right")
    cnt = hi - lo
    total = int(cnt.sum())
    jj = np.repeat(np.arange(len(sk), dtype=np.int64), cnt)
    start = np.repeat(lo, cnt)
    within = np.arange(total, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    ii = qpos[start + within]
    return ii, jj, qi, stride


def _f32log2(x: int) -> np.float32:
    return np.float32(np.log2(np.float32(x))) * np.float32(1.0 / 16.0)


def _ratio(a: int, b: int) -> np.float32:
    return np.float32(a) / np.float32(b) if b else np.float32(0.0)


def pair_features(q, s) -> np.ndarray:
    """The 32 features of one pair (see the module docstring)."""
    q = np.asarray(q, dtype=np.int64)
    s = np.asarray(s, dtype=np.int64)
    m, n = len(q), len(s)
    f = np.zeros(NFEAT, dtype=np.float32)
    f[0] = _f32log2(1 + m)
    f[1] = _f32log2(1 + n)
    f[2] = _f32log2(1 + abs(n - m))
    f[3] = _ratio(min(m, n), max(m, n))
    ii, jj, qi, stride = hits(q, s)
    nq = max(0, m - KMER + 1)
    ns = len(qi)
    H = len(ii)
    matched = np.unique(ii)
    f[4] = _ratio(len(matched), ns)
    f[5] = _f32log2(1 + H)
    if nq > 0:
        seg_all = (NSEG * qi) // nq
        seg_hit = (NSEG * matched) // nq
        for k in range(NSEG):
            f[6 + k] = _ratio(int((seg_hit == k).sum()), int((seg_all == k).sum()))
    if H:
        d = jj - ii
        dlo, dhi = min(0, n - m), max(0, n - m)
        e = d - np.clip(d, dlo, dhi)
        a = np.abs(e)
        bl = np.frexp(a.astype(np.float64))[1].astype(np.int64)  # bit length (0 for a = 0)
        b = np.minimum(bl, NBINS - 1)
        cnt = np.bincount(b, minlength=NBINS)
        for k in range(NBINS):
            f[14 + k] = _ratio(int(cnt[k]), H)
        f[30] = _ratio(int((e < 0).sum()), H)
    f[31] = np.float32(1.0) / np.float32(stride)
    return f


def batch_features(q_codes, q_off, t_codes, t_off) -> np.ndarray:
    """Features of pairs p = (q_p, t_p) in CSR form: float32[npairs, 32]."""
    npairs = len(q_off) - 1
    out = np.zeros((npairs, NFEAT), dtype=np.float32)
    for p in range(npairs):
        out[p] = pair_features(q_codes[q_off[p]:q_off[p + 1]], t_codes[t_off[p]:t_off[p + 1]])
    return out
