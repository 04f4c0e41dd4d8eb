"""Brute-force alignment enumerator -- TEST INFRASTRUCTURE (pins the DP oracle).

Independent of the dynamic programme: it lists every alignment of two short
sequences explicitly as a string of columns (M: q_i over s_j, D: q_i over a
gap, I: s_j over a gap) and scores it directly from the definitions of
Sec. 2.1 of the AnySeq/GPU paper:

* substitution score sigma(q_i, s_j) for every M column;
* a maximal run of k gap columns of the same kind costs alpha + (k-1)*beta
  ("Affine Gap Penalty"); a D run next to an I run are two runs, each
  paying alpha (the recurrence lets H(i,j) come from F and feed E).

Modes, from the paragraphs "Local/Global/Semi-global Alignments":

* global      -- max over all alignments of q against s;
* local       -- max(0, max over all substring pairs of their global score);
* semi-global -- max over alignments of q[i0:i1] vs s[j0:j1] whose start
                 lies on row 0 or column 0 (i0 == 0 or j0 == 0) and whose end
                 lies on row m or column n (i1 == m or j1 == n): gaps at both
                 ends of both sequences are free.

The number of alignments of lengths (a, b) is the Delannoy number D(a, b)
(D(6,6) = 8989), so this is only usable for lengths up to about 6.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np


@functools.lru_cache(maxsize=None)
def alignments(a: int, b: int) -> tuple:
    """All alignments of lengths (a, b) as tuples of 'M', 'D', 'I'."""
    if a == 0 and b == 0:
        return ((),)
    out = []
    if a > 0 and b > 0:
        out += [x + ("M",) for x in alignments(a - 1, b - 1)]
    if a > 0:
        out += [x + ("D",) for x in alignments(a - 1, b)]
    if b > 0:
        out += [x + ("I",) for x in alignments(a, b - 1)]
    return tuple(out)


def delannoy(a: int, b: int) -> int:
    return len(alignments(a, b))


@functools.lru_cache(maxsize=None)
def _tables(a: int, b: int):
    """For every alignment: indicator of matched (i, j), #gap runs, #gap residues."""
    al = alignments(a, b)
    K = len(al)
    match = np.zeros((K, max(a, 1), max(b, 1)), dtype=np.int64)
    runs = np.zeros(K, dtype=np.int64)
    gaps = np.zeros(K, dtype=np.int64)
    for k, ops in enumerate(al):
        i = j = 0
        prev = None
        for op in ops:
            if op == "M":
                match[k, i, j] = 1
                i += 1
                j += 1
            else:
                gaps[k] += 1
                if op != prev:
                    runs[k] += 1
                if op == "D":
                    i += 1
                else:
                    j += 1
            prev = op
    return match, runs, gaps


def score_alignment(ops, q, s, sigma, alpha, beta) -> int:
    """Score of one explicit alignment (used by the hand-worked tests)."""
    i = j = 0
    total = 0
    prev = None
    for op in ops:
        if op == "M":
            total += int(sigma[q[i]][s[j]])
            i += 1
            j += 1
        else:
            total -= beta if op == prev else alpha
            if op == "D":
                i += 1
            else:
                j += 1
        prev = op
    assert i == len(q) and j == len(s)
    return total


def global_scores(q, s, sigma, alpha, beta) -> np.ndarray:
    """Scores of every alignment of q against s (vector over alignments)."""
    a, b = len(q), len(s)
    match, runs, gaps = _tables(a, b)
    gap_cost = alpha * runs + beta * (gaps - runs)
    if a == 0 or b == 0:
        return -gap_cost
    sig = np.asarray(sigma, dtype=np.int64)[np.ix_(np.asarray(q), np.asarray(s))]
    return np.einsum("kij,ij->k", match, sig) - gap_cost


def global_table(Q: np.ndarray, S: np.ndarray, sigma, alpha, beta, chunk: int = 32) -> np.ndarray:
    """Brute-force global scores of every pair of rows of Q (Nq x a codes)
    and S (Ns x b codes), all of one length pair (a, b): the same explicit
    alignment list as global_scores, scored for many pairs at once.
    Returns an (Nq, Ns) int64 table."""
    Q = np.asarray(Q, dtype=np.int64).reshape(len(Q), -1)
    S = np.asarray(S, dtype=np.int64).reshape(len(S), -1)
    a, b = Q.shape[1], S.shape[1]
    match, runs, gaps = _tables(a, b)
    gap_cost = alpha * runs + beta * (gaps - runs)
    out = np.empty((len(Q), len(S)), dtype=np.int64)
    if a == 0 or b == 0:
        out[:] = -int(gap_cost.min())  # one alignment: every column a gap
        return out
    sig = np.asarray(sigma, dtype=np.int64)
    mflat = match.reshape(len(match), a * b).T  # (a*b, K)
    for c0 in range(0, len(Q), chunk):
        qc = Q[c0:c0 + chunk]
        # sigma(q_i, s_j) for every pair of the chunk: (nq, Ns, a, b)
        pair_sig = sig[qc[:, None, :, None], S[None, :, None, :]]
        scores = pair_sig.reshape(len(qc) * len(S), a * b) @ mflat - gap_cost[None, :]
        out[c0:c0 + chunk] = scores.max(axis=1).reshape(len(qc), len(S))
    return out


def brute_global(q, s, sigma, alpha, beta) -> int:
    return int(global_scores(q, s, sigma, alpha, beta).max())


def brute_local(q, s, sigma, alpha, beta) -> int:
    m, n = len(q), len(s)
    best = 0
    for i0, i1 in itertools.combinations_with_replacement(range(m + 1), 2):
        for j0, j1 in itertools.combinations_with_replacement(range(n + 1), 2):
            best = max(best, brute_global(q[i0:i1], s[j0:j1], sigma, alpha, beta))
    return best


def brute_semiglobal(q, s, sigma, alpha, beta) -> int:
    m, n = len(q), len(s)
    best = None
    for i0 in range(m + 1):
        for j0 in range(n + 1):
            if i0 != 0 and j0 != 0:
                continue
            for i1 in range(i0, m + 1):
                for j1 in range(j0, n + 1):
                    if i1 != m and j1 != n:
                        continue
                    v = brute_global(q[i0:i1], s[j0:j1], sigma, alpha, beta)
                    best = v if best is None else max(best, v)
    return best


def brute(q, s, sigma, alpha, beta, mode) -> int:
    mode = {"local": 0, "global": 1, "semiglobal": 2, "semi": 2}.get(mode, mode)
    if mode == 0:
        return brute_local(q, s, sigma, alpha, beta)
    if mode == 1:
        return brute_global(q, s, sigma, alpha, beta)
    return brute_semiglobal(q, s, sigma, alpha, beta)


def brute_banded_global(q, s, sigma, alpha, beta, lo, hi) -> int | None:
    """Best global alignment whose path stays on diagonals lo <= j - i <= hi
    (every visited lattice point, including (0,0) and (m,n)); None if none."""
    a, b = len(q), len(s)
    al = alignments(a, b)
    scores = global_scores(q, s, sigma, alpha, beta)
    best = None
    for k, ops in enumerate(al):
        i = j = 0
        ok = lo <= 0 <= hi
        for op in ops:
            if op in "MD":
                i += 1
            if op in "MI":
                j += 1
            if not (lo <= j - i <= hi):
                ok = False
                break
        if ok:
            v = int(scores[k])
            best = v if best is None else max(best, v)
    return best
