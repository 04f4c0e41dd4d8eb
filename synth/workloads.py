"""Seeded synthetic alignment workloads (inputs only; no alignment arithmetic).

All generators draw from ``numpy.random.Generator(PCG64(seed))`` and are
vectorised over the whole batch (processed in chunks of pairs so that the
1M-pair batch fits in a few hundred MB).  The five workloads mirror the
shapes of the paper's read sets (Sec. 4.1: read lengths 125..4096, long
PacBio-like reads) and of the five benchmark configurations:

1. ``uniform_dna_pairs``   -- 1,000 pairs of 150 vs 150 uniform ACGT.
2. ``mutated_dna_pairs``   -- 1M pairs, |Q| ~ U{100..300}; S = Q with 5 %
   substitutions (uniform among the other three bases) and 1 % indel events
   (50/50 insertion/deletion, length ~ Geometric(p=0.5) on {1,2,...}, mean 2;
   inserted bases uniform).
3. ``protein_database``    -- 512 queries |Q| ~ U{100..1000} against 200k
   targets |T| ~ LogNormal(ln 300, 0.6) redrawn outside [10, 5000]; residues
   i.i.d. from the BLOSUM62 background frequencies.
4. ``long_dna_pairs``      -- 20k pairs |Q| ~ U{1000..20000}; per pair
   divergence d ~ U(1 %, 15 %), indel fraction f ~ U(10 %, 40 %) of events,
   indel length Geometric(mean 2).
5. ``serving_stream``      -- Poisson arrivals, lengths LogNormal(median
   1000, sigma 1.2) clipped to [100, 50000], 60 % DNA (model 2) / 40 %
   protein (85 %-identity copy), 50/50 local/global.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .tables import PROTEIN_BACKGROUND, blosum62, dna_matrix

SEED_BASE = 20220607


@dataclasses.dataclass
class Batch:
    """Pairs p = (q_p, t_p) in CSR form: codes[off[p]:off[p+1]]."""
    q_codes: np.ndarray
    q_off: np.ndarray
    t_codes: np.ndarray
    t_off: np.ndarray
    matrix: np.ndarray
    alpha: int
    beta: int
    name: str = ""
    seed: int = 0

    @property
    def npairs(self) -> int:
        return len(self.q_off) - 1

    def lengths(self):
        return np.diff(self.q_off), np.diff(self.t_off)

    def cells(self) -> int:
        m, n = self.lengths()
        return int(np.sum(m.astype(np.int64) * n.astype(np.int64)))

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        q = [self.q_codes[self.q_off[i]:self.q_off[i + 1]] for i in idx]
        t = [self.t_codes[self.t_off[i]:self.t_off[i + 1]] for i in idx]
        qc, qo = pack_csr(q)
        tc, to = pack_csr(t)
        return Batch(qc, qo, tc, to, self.matrix, self.alpha, self.beta, self.name + "[subset]",
                     self.seed)


@dataclasses.dataclass
class CrossBatch:
    """All-vs-all: nq queries x nt targets."""
    q_codes: np.ndarray
    q_off: np.ndarray
    t_codes: np.ndarray
    t_off: np.ndarray
    matrix: np.ndarray
    alpha: int
    beta: int
    name: str = ""
    seed: int = 0

    @property
    def nq(self) -> int:
        return len(self.q_off) - 1

    @property
    def nt(self) -> int:
        return len(self.t_off) - 1

    def cells(self) -> int:
        return int(np.sum(np.diff(self.q_off))) * int(np.sum(np.diff(self.t_off)))


@dataclasses.dataclass
class Stream:
    """Serving requests: arrival time (s), pair, alphabet (0 DNA, 1 protein), mode."""
    arrival: np.ndarray
    q_codes: np.ndarray
    q_off: np.ndarray
    t_codes: np.ndarray
    t_off: np.ndarray
    protein: np.ndarray
    mode: np.ndarray
    dna_scoring: tuple
    protein_scoring: tuple
    seed: int = 0

    @property
    def nreq(self) -> int:
        return len(self.arrival)


def pack_csr(seqs):
    """List of code arrays -> (codes uint8, offsets int64)."""
    lens = np.array([len(s) for s in seqs], dtype=np.int64)
    off = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    codes = np.concatenate([np.asarray(s, dtype=np.uint8) for s in seqs]) if len(seqs) and off[-1] \
        else np.zeros(0, dtype=np.uint8)
    return codes, off


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_sequences(rng, lengths, alphabet_size=4, freqs=None):
    """Concatenated i.i.d. residues for the given lengths -> (codes, off)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    total = int(off[-1])
    if freqs is None:
        codes = rng.integers(0, alphabet_size, size=total, dtype=np.uint8)
    else:
        cdf = np.cumsum(freqs)
        cdf[-1] = 1.0
        codes = np.searchsorted(cdf, rng.random(total), side="right").astype(np.uint8)
    return codes, off


def mutate(rng, codes, off, p_event, indel_frac, alphabet_size=4, freqs=None,
           chunk_residues=1 << 23):
    """Mutated copies of the sequences codes[off[k]:off[k+1]].

    Per position an event happens with probability p_event[k]; an event is an
    indel with probability indel_frac[k] (50/50 insertion before the position
    or deletion starting at it, length ~ Geometric(0.5) on {1,2,...},
    deletions clipped at the sequence end), otherwise a substitution by a
    different residue (uniform among the others, or drawn from ``freqs``
    conditioned on differing).  Returns (codes, off) of the copies.  The
    sequences are processed in groups of about chunk_residues residues.
    """
    nseq = len(off) - 1
    pe = np.broadcast_to(np.asarray(p_event, dtype=np.float64), (nseq,))
    fi = np.broadcast_to(np.asarray(indel_frac, dtype=np.float64), (nseq,))
    outs, lens = [], []
    k = 0
    while k < nseq:
        k2 = int(np.searchsorted(off, off[k] + chunk_residues, side="right")) - 1
        k2 = min(max(k2, k + 1), nseq)
        sub_off = off[k:k2 + 1] - off[k]
        c, o = _mutate_core(rng, codes[off[k]:off[k2]], sub_off, pe[k:k2], fi[k:k2], alphabet_size,
                            freqs)
        outs.append(c)
        lens.append(np.diff(o))
        k = k2
    if not outs:
        return np.zeros(0, dtype=np.uint8), np.zeros(nseq + 1, dtype=np.int64)
    new_off = np.zeros(nseq + 1, dtype=np.int64)
    np.cumsum(np.concatenate(lens), out=new_off[1:])
    return np.concatenate(outs), new_off


def _mutate_core(rng, codes, off, pe, fi, alphabet_size, freqs):
    nseq = len(off) - 1
    lens = np.diff(off)
    N = int(off[-1])
    seq_id = np.repeat(np.arange(nseq, dtype=np.int64), lens)
    event = rng.random(N, dtype=np.float32) < pe.astype(np.float32)[seq_id]
    eidx = np.nonzero(event)[0]
    is_indel = rng.random(len(eidx)) < fi[seq_id[eidx]]
    is_ins = rng.random(len(eidx)) < 0.5
    sidx = eidx[~is_indel]
    iidx = eidx[is_indel & is_ins]
    didx = eidx[is_indel & ~is_ins]
    ilen = rng.geometric(0.5, size=len(iidx)).astype(np.int64)
    dlen = rng.geometric(0.5, size=len(didx)).astype(np.int64)

    out = codes.copy()
    # substitutions
    if len(sidx):
        if freqs is None:
            shift = rng.integers(1, alphabet_size, size=len(sidx))
            out[sidx] = ((out[sidx].astype(np.int64) + shift) % alphabet_size).astype(np.uint8)
        else:
            cdf = np.cumsum(freqs)
            cdf[-1] = 1.0
            new = np.searchsorted(cdf, rng.random(len(sidx)), side="right").astype(np.uint8)
            same = new == out[sidx]
            while np.any(same):
                new[same] = np.searchsorted(cdf, rng.random(int(same.sum())), side="right")
                same = new == out[sidx]
            out[sidx] = new
    # deletions: positions [x, min(x+L, end)) removed
    diff = np.zeros(N + 1, dtype=np.int32)
    if len(didx):
        ends = np.minimum(didx + dlen, off[seq_id[didx] + 1])
        np.add.at(diff, didx, 1)
        np.add.at(diff, ends, -1)
    per_pos = (np.cumsum(diff[:N]) == 0).astype(np.int64)  # kept residues
    per_pos[iidx] += ilen                                    # insertions before the position
    ins_count = np.zeros(N, dtype=np.int64)
    ins_count[iidx] = ilen
    total = int(per_pos.sum())
    start = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(per_pos, out=start[1:])
    src = np.repeat(np.arange(N, dtype=np.int64), per_pos)
    rank = np.arange(total, dtype=np.int64) - start[src]
    is_new = rank < ins_count[src]
    new = np.empty(total, dtype=np.uint8)
    n_ins = int(is_new.sum())
    if freqs is None:
        new[is_new] = rng.integers(0, alphabet_size, size=n_ins, dtype=np.uint8)
    else:
        cdf = np.cumsum(freqs)
        cdf[-1] = 1.0
        new[is_new] = np.searchsorted(cdf, rng.random(n_ins), side="right").astype(np.uint8)
    new[~is_new] = out[src[~is_new]]
    out_len = start[off[1:]] - start[off[:-1]]
    new_off = np.zeros(nseq + 1, dtype=np.int64)
    np.cumsum(out_len, out=new_off[1:])
    return new, new_off


def uniform_dna_pairs(npairs=1000, m=150, n=150, seed=SEED_BASE + 1, match=2, mismatch=-3,
                      alpha=5, beta=2) -> Batch:
    """Configuration 1: independent uniform ACGT pairs of fixed lengths."""
    rng = _rng(seed)
    qc, qo = random_sequences(rng, np.full(npairs, m))
    tc, to = random_sequences(rng, np.full(npairs, n))
    return Batch(qc, qo, tc, to, dna_matrix(match, mismatch), alpha, beta,
                 f"dna-uniform-{npairs}x{m}x{n}", seed)


def mutated_dna_pairs(npairs=1_000_000, lmin=100, lmax=300, sub=0.05, indel=0.01,
                      seed=SEED_BASE + 2, match=2, mismatch=-3, alpha=5, beta=2,
                      chunk=200_000) -> Batch:
    """Configuration 2: S = mutated copy of Q (5 % substitutions, 1 % indels)."""
    rng = _rng(seed)
    qs, ts, qo_parts, to_parts = [], [], [], []
    done = 0
    while done < npairs:
        k = min(chunk, npairs - done)
        lens = rng.integers(lmin, lmax + 1, size=k)
        qc, qo = random_sequences(rng, lens)
        p_event = sub + indel
        tc, to = mutate(rng, qc, qo, p_event, indel / p_event)
        qs.append(qc); ts.append(tc); qo_parts.append(qo); to_parts.append(to)
        done += k
    return Batch(*_merge(qs, qo_parts), *_merge(ts, to_parts), dna_matrix(match, mismatch),
                 alpha, beta, f"dna-mutated-{npairs}-{lmin}-{lmax}", seed)


def _merge(codes_list, off_list):
    codes = np.concatenate(codes_list) if codes_list else np.zeros(0, np.uint8)
    offs = [np.zeros(1, dtype=np.int64)]
    base = 0
    for o in off_list:
        offs.append(o[1:] + base)
        base += int(o[-1])
    return codes, np.concatenate(offs)


def _lognormal_lengths(rng, k, median, sigma, lo, hi):
    out = np.empty(k, dtype=np.int64)
    todo = np.arange(k)
    while len(todo):
        x = np.rint(rng.lognormal(np.log(median), sigma, size=len(todo))).astype(np.int64)
        ok = (x >= lo) & (x <= hi)
        out[todo[ok]] = x[ok]
        todo = todo[~ok]
    return out


def protein_database(nq=512, qmin=100, qmax=1000, nt=200_000, median=300, sigma=0.6,
                     tmin=10, tmax=5000, seed=SEED_BASE + 3, alpha=11, beta=1) -> CrossBatch:
    """Configuration 3: queries x database, i.i.d. background residues, BLOSUM62."""
    rng = _rng(seed)
    qlens = rng.integers(qmin, qmax + 1, size=nq)
    tlens = _lognormal_lengths(rng, nt, median, sigma, tmin, tmax)
    qc, qo = random_sequences(rng, qlens, 24, np.concatenate([PROTEIN_BACKGROUND, np.zeros(4)]))
    tc, to = random_sequences(rng, tlens, 24, np.concatenate([PROTEIN_BACKGROUND, np.zeros(4)]))
    return CrossBatch(qc, qo, tc, to, blosum62(), alpha, beta,
                      f"protein-db-{nq}x{nt}", seed)


def long_dna_pairs(npairs=20_000, lmin=1000, lmax=20000, dmin=0.01, dmax=0.15, fmin=0.10,
                   fmax=0.40, seed=SEED_BASE + 4, match=2, mismatch=-3, alpha=5, beta=2,
                   chunk=2000) -> Batch:
    """Configuration 4: long global pairs with per-pair divergence/indel mix."""
    rng = _rng(seed)
    qs, ts, qo_parts, to_parts = [], [], [], []
    done = 0
    while done < npairs:
        k = min(chunk, npairs - done)
        lens = rng.integers(lmin, lmax + 1, size=k)
        d = rng.uniform(dmin, dmax, size=k)
        f = rng.uniform(fmin, fmax, size=k)
        qc, qo = random_sequences(rng, lens)
        tc, to = mutate(rng, qc, qo, d, f)
        qs.append(qc); ts.append(tc); qo_parts.append(qo); to_parts.append(to)
        done += k
    return Batch(*_merge(qs, qo_parts), *_merge(ts, to_parts), dna_matrix(match, mismatch),
                 alpha, beta, f"dna-long-{npairs}-{lmin}-{lmax}", seed)


def _interleave(n, parts):
    """Merge CSR sets whose sequences belong to request indices idx into one
    CSR in request order."""
    lens = np.zeros(n, dtype=np.int64)
    for idx, _, off in parts:
        lens[idx] = np.diff(off)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    out = np.empty(int(out_off[-1]), dtype=np.uint8)
    for idx, codes, off in parts:
        ln = np.diff(off)
        tot = int(ln.sum())
        if not tot:
            continue
        # destination of every residue: request start + position in request
        dst = np.repeat(out_off[idx] - off[:-1], ln) + np.arange(off[0], off[0] + tot)
        out[dst] = codes[off[0]:off[0] + tot]
    return out, out_off


def serving_stream(nreq=200_000, rate=1.0e4, median=1000, sigma=1.2, lmin=100, lmax=50_000,
                   frac_dna=0.6, seed=SEED_BASE + 5) -> Stream:
    """Configuration 5: Poisson request stream of mixed DNA/protein pairs."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate, size=nreq)
    arrival = np.cumsum(gaps)
    lens = np.clip(np.rint(rng.lognormal(np.log(median), sigma, size=nreq)), lmin, lmax).astype(np.int64)
    protein = rng.random(nreq) >= frac_dna
    mode = np.where(rng.random(nreq) < 0.5, 0, 1).astype(np.int32)  # 0 local, 1 global
    bg = np.concatenate([PROTEIN_BACKGROUND, np.zeros(4)])
    parts = []  # (request indices, q CSR, t CSR) per alphabet
    for is_prot in (False, True):
        idx = np.nonzero(protein == is_prot)[0]
        if not len(idx):
            continue
        if is_prot:
            qc, qo = random_sequences(rng, lens[idx], 24, bg)
            tc, to = mutate(rng, qc, qo, 0.15, 0.1, 24, bg)
        else:
            qc, qo = random_sequences(rng, lens[idx])
            tc, to = mutate(rng, qc, qo, 0.06, 1.0 / 6.0)
        parts.append((idx, qc, qo, tc, to))
    qc, qo = _interleave(nreq, [(p[0], p[1], p[2]) for p in parts])
    tc, to = _interleave(nreq, [(p[0], p[3], p[4]) for p in parts])
    return Stream(arrival, qc, qo, tc, to, protein, mode, (dna_matrix(2, -3), 5, 2),
                  (blosum62(), 11, 1), seed)
