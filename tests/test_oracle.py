"""Pins of the CPU oracle against things other than itself (no GPU).

* brute force: every alignment enumerated and scored from the definitions
  (oracle/brute.py), exhaustively for every pair of DNA strings of length
  0..4 and on random DNA and protein inputs up to length 6;
* closed forms: identical sequences, one empty sequence, AAAA vs CCCC;
* an independent linear-gap DP (the paper's linear scheme) equals the affine
  oracle at alpha == beta;
* invariants: mode ordering, non-negativity, symmetry with the transposed
  matrix, monotonicity in the gap costs, superadditivity of global scores,
  monotonicity of local scores under extension;
* hand-worked DP tables (tests/golden/hand_worked.json);
* banded DP against path-restricted brute force, and the band certificate
  against the full DP.
A planted mistake (dropped term, wrong sign, swapped operand) in the oracle
fails at least one of these.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = ["local", "global", "semiglobal"]
SCHEMES = [((2, -3), 5, 2), ((1, -1), 2, 1), ((2, -1), 2, 2), ((3, -2), 4, 1)]


def _dna(rng, n):
    return rng.integers(0, 4, size=n).astype(np.uint8)


def _prot(rng, n):
    return rng.integers(0, 20, size=n).astype(np.uint8)


def test_delannoy_count():
    # number of alignments of (6,6) is the Delannoy number D(6,6) = 8989
    assert brute.delannoy(6, 6) == 8989
    assert brute.delannoy(3, 3) == 63


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scheme", SCHEMES[:2])
def test_exhaustive_short_dna(mode, scheme):
    (ma, mi), alpha, beta = scheme
    sig = synth.dna_matrix(ma, mi)
    seqs = [np.array(s, dtype=np.uint8) for L in range(0, 3)
            for s in itertools.product(range(4), repeat=L)]
    for q in seqs:
        for s in seqs:
            assert oracle.score(q, s, sig, alpha, beta, mode) == \
                brute.brute(q, s, sig, alpha, beta, mode), (q, s, mode)


ASYM = np.array([[3, -2, -4, 1], [-1, 2, -3, -2], [0, -4, 4, -1], [-3, 1, -2, 2]], dtype=np.int8)


@pytest.mark.parametrize("scheme", SCHEMES[:2] + [(ASYM, 3, 1)])
def test_exhaustive_dna_up_to_4(scheme):
    """Every pair of DNA strings of length 0..4 (341 strings, 116,281 pairs),
    all three modes: the C oracle against brute force.  Global scores of
    every pair of strings come from the explicit alignment enumeration
    (vectorised over pairs); local and semi-global follow from them by their
    definitions over substrings (Sec. 2.1): local = max(0, max over substring
    pairs), semi-global = max over substrings that start on row or column 0
    and end on row m or column n."""
    mat, alpha, beta = scheme  # (match, mismatch) or an asymmetric 4 x 4 matrix (sigma(q, s) != sigma(s, q))
    sig = mat if isinstance(mat, np.ndarray) else synth.dna_matrix(*mat)
    by_len = [np.array(list(itertools.product(range(4), repeat=L)), dtype=np.uint8).reshape(4 ** L, L)
              for L in range(5)]
    base = np.cumsum([0] + [len(x) for x in by_len])  # id of string k of length L: base[L] + k
    nstr = int(base[-1])
    G = np.empty((nstr, nstr), dtype=np.int64)
    for a in range(5):
        for b in range(5):
            G[base[a]:base[a + 1], base[b]:base[b + 1]] = brute.global_table(by_len[a], by_len[b], sig, alpha,
                                                                           beta)

    def sid(x):  # id of a code string
        k = 0
        for c in x:
            k = 4 * k + int(c)
        return int(base[len(x)]) + k

    want = {m: np.empty((nstr, nstr), dtype=np.int64) for m in MODES}
    for a in range(5):
        for b in range(5):
            qa, sb = by_len[a], by_len[b]
            # substring ids of every string of the two lengths
            subq = [(i0, i1) for i0 in range(a + 1) for i1 in range(i0, a + 1)]
            subs = [(j0, j1) for j0 in range(b + 1) for j1 in range(j0, b + 1)]
            Iq = np.array([[sid(x[i0:i1]) for (i0, i1) in subq] for x in qa])  # (Nq, nsubq)
            Is = np.array([[sid(y[j0:j1]) for (j0, j1) in subs] for y in sb])  # (Ns, nsubs)
            loc = np.zeros((len(qa), len(sb)), dtype=np.int64)
            semi = np.full((len(qa), len(sb)), np.iinfo(np.int64).min, dtype=np.int64)
            for u, (i0, i1) in enumerate(subq):
                for v, (j0, j1) in enumerate(subs):
                    g = G[Iq[:, u][:, None], Is[:, v][None, :]]
                    loc = np.maximum(loc, g)
                    if (i0 == 0 or j0 == 0) and (i1 == a or j1 == b):
                        semi = np.maximum(semi, g)
            sl = (slice(base[a], base[a + 1]), slice(base[b], base[b + 1]))
            want["global"][sl] = G[sl]
            want["local"][sl] = loc
            want["semiglobal"][sl] = semi
    strings = [x for L in range(5) for x in by_len[L]]
    qc, qo = synth.pack_csr([x for x in strings for _ in strings])
    tc, to = synth.pack_csr([y for _ in strings for y in strings])
    for mode in MODES:
        got, errs = oracle.batch(qc, qo, tc, to, sig, alpha, beta, mode, nthreads=4)
        assert not errs.any()
        bad = np.nonzero(got != want[mode].ravel())[0]
        assert len(bad) == 0, (mode, bad[:5])


@pytest.mark.parametrize("mode", MODES)
def test_random_dna_vs_brute(mode):
    rng = np.random.default_rng(11 + MODES.index(mode))
    for k in range(60):
        (ma, mi), alpha, beta = SCHEMES[k % len(SCHEMES)]
        sig = synth.dna_matrix(ma, mi)
        m, n = rng.integers(0, 6, size=2) if mode != "global" else rng.integers(0, 7, size=2)
        q, s = _dna(rng, m), _dna(rng, n)
        assert oracle.score(q, s, sig, alpha, beta, mode) == brute.brute(q, s, sig, alpha, beta, mode)


@pytest.mark.parametrize("mode", MODES)
def test_random_protein_vs_brute(mode):
    rng = np.random.default_rng(23 + MODES.index(mode))
    sig = synth.blosum62()
    for _ in range(25):
        m, n = rng.integers(1, 5, size=2)
        q, s = _prot(rng, m), _prot(rng, n)
        assert oracle.score(q, s, sig, 11, 1, mode) == brute.brute(q, s, sig, 11, 1, mode)
        assert oracle.score(q, s, sig, 4, 2, mode) == brute.brute(q, s, sig, 4, 2, mode)


def test_asymmetric_matrix_vs_brute():
    # a non-symmetric sigma catches a transposed q/s operand
    rng = np.random.default_rng(5)
    sig = rng.integers(-4, 5, size=(4, 4)).astype(np.int8)
    for mode in MODES:
        for _ in range(20):
            m, n = rng.integers(0, 5, size=2)
            q, s = _dna(rng, m), _dna(rng, n)
            assert oracle.score(q, s, sig, 3, 1, mode) == brute.brute(q, s, sig, 3, 1, mode)


def test_closed_forms():
    sig = synth.dna_matrix(2, -3)
    rng = np.random.default_rng(3)
    for n in (1, 5, 37, 150):
        q = _dna(rng, n)
        for mode in MODES:
            assert oracle.score(q, q, sig, 5, 2, mode) == 2 * n
        # global against an empty sequence: one gap run of length n
        e = np.zeros(0, dtype=np.uint8)
        assert oracle.score(q, e, sig, 5, 2, "global") == -5 - 2 * (n - 1)
        assert oracle.score(e, q, sig, 5, 2, "global") == -5 - 2 * (n - 1)
        assert oracle.score(q, e, sig, 5, 2, "local") == 0
        assert oracle.score(q, e, sig, 5, 2, "semiglobal") == 0
    e = np.zeros(0, dtype=np.uint8)
    for mode in MODES:
        assert oracle.score(e, e, sig, 5, 2, mode) == 0
    a = synth.encode("AAAA")
    c = synth.encode("CCCC")
    assert oracle.score(a, c, sig, 5, 2, "global") == -12


def _linear_gap_dp(q, s, sig, g, mode):
    """The paper's linear-gap scheme: E = H(i-1,j) - g, F = H(i,j-1) - g."""
    m, n = len(q), len(s)
    glob = mode == "global"
    H = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        H[i, 0] = -g * i if glob else 0
    for j in range(1, n + 1):
        H[0, j] = -g * j if glob else 0
    nu = 0 if mode == "local" else -(10 ** 12)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            H[i, j] = max(H[i - 1, j - 1] + int(sig[q[i - 1]][s[j - 1]]), H[i - 1, j] - g,
                          H[i, j - 1] - g, nu)
    if mode == "global":
        return int(H[m, n])
    if mode == "local":
        return int(max(0, H.max()))
    return int(max(H[m, :].max(), H[:, n].max()))


@pytest.mark.parametrize("mode", MODES)
def test_alpha_eq_beta_is_linear_gap(mode):
    rng = np.random.default_rng(7)
    sig = synth.dna_matrix(2, -1)
    for _ in range(40):
        m, n = rng.integers(0, 40, size=2)
        q, s = _dna(rng, m), _dna(rng, n)
        for g in (1, 3):
            assert oracle.score(q, s, sig, g, g, mode) == _linear_gap_dp(q, s, sig, g, mode)


def test_invariants():
    rng = np.random.default_rng(17)
    for alph, sig, (al, be) in ((4, synth.dna_matrix(2, -3), (5, 2)),
                                (20, synth.blosum62(), (11, 1))):
        for _ in range(30):
            m, n = rng.integers(0, 60, size=2)
            q = rng.integers(0, alph, size=m).astype(np.uint8)
            s = rng.integers(0, alph, size=n).astype(np.uint8)
            loc = oracle.score(q, s, sig, al, be, "local")
            sem = oracle.score(q, s, sig, al, be, "semiglobal")
            glo = oracle.score(q, s, sig, al, be, "global")
            assert loc >= sem >= glo
            assert loc >= 0 and sem >= 0
            sigT = np.ascontiguousarray(np.asarray(sig).T)
            for mode, v in (("local", loc), ("semiglobal", sem), ("global", glo)):
                assert oracle.score(s, q, sigT, al, be, mode) == v
                assert oracle.score(q, s, sig, al + 1, be, mode) <= v
                assert oracle.score(q, s, sig, al + 1, be + 1, mode) <= v
            # superadditivity of global scores over a split
            if m >= 2 and n >= 2:
                a, b = int(rng.integers(1, m)), int(rng.integers(1, n))
                assert glo >= oracle.score(q[:a], s[:b], sig, al, be, "global") + \
                    oracle.score(q[a:], s[b:], sig, al, be, "global")
            # local never drops when a sequence grows
            extra = rng.integers(0, alph, size=5).astype(np.uint8)
            assert oracle.score(np.concatenate([q, extra]), s, sig, al, be, "local") >= loc
            assert oracle.score(q, np.concatenate([extra, s]), sig, al, be, "local") >= loc


def test_hand_worked_tables():
    data = json.load(open(os.path.join(GOLDEN, "hand_worked.json")))
    for c in data["cases"]:
        sig = synth.dna_matrix(c["match"], c["mismatch"])
        q, s = synth.encode(c["query"]), synth.encode(c["target"])
        sc, H = oracle.score_matrix(q, s, sig, c["alpha"], c["beta"], c["mode"])
        assert sc == c["score"], c["name"]
        assert oracle.score(q, s, sig, c["alpha"], c["beta"], c["mode"]) == c["score"]
        assert brute.brute(q, s, sig, c["alpha"], c["beta"], c["mode"]) == c["score"]
        if "H" in c:
            assert (H == np.array(c["H"])).all(), c["name"]


def test_unread_borders_reading():
    # E(i,0) and F(0,j) are printed in the init tables but no cell reads them
    rng = np.random.default_rng(2)
    sig = synth.dna_matrix(2, -3)
    for _ in range(20):
        q, s = _dna(rng, rng.integers(0, 30)), _dna(rng, rng.integers(0, 30))
        for mode in MODES:
            assert oracle.score(q, s, sig, 5, 2, mode, flags=1) == oracle.score(q, s, sig, 5, 2, mode)


def test_residue_error():
    sig = synth.dna_matrix(2, -3)
    with pytest.raises(oracle.OracleError):
        oracle.score(np.array([0, 4], np.uint8), np.array([1], np.uint8), sig, 5, 2, "local")


def test_batch_and_cross_runners():
    b = synth.uniform_dna_pairs(npairs=40, m=30, n=25, seed=9)
    for mode in MODES:
        out, errs = oracle.batch(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, 5, 2, mode,
                                 nthreads=3)
        assert not errs.any()
        for p in range(b.npairs):
            q = b.q_codes[b.q_off[p]:b.q_off[p + 1]]
            t = b.t_codes[b.t_off[p]:b.t_off[p + 1]]
            assert out[p] == oracle.score(q, t, b.matrix, 5, 2, mode)
    cr = synth.protein_database(nq=3, qmin=5, qmax=20, nt=7, median=15, seed=4)
    out, errs = oracle.cross(cr.q_codes, cr.q_off, cr.t_codes, cr.t_off, cr.matrix, 11, 1, "local",
                             nthreads=2)
    for i in range(cr.nq):
        for j in range(cr.nt):
            q = cr.q_codes[cr.q_off[i]:cr.q_off[i + 1]]
            t = cr.t_codes[cr.t_off[j]:cr.t_off[j + 1]]
            assert out[i, j] == oracle.score(q, t, cr.matrix, 11, 1, "local")


# ---------------------------------------------------------------- banded
def test_banded_vs_path_restricted_brute():
    rng = np.random.default_rng(31)
    sig = synth.dna_matrix(2, -3)
    for _ in range(60):
        m, n = rng.integers(0, 6, size=2)
        q, s = _dna(rng, m), _dna(rng, n)
        dn = n - m
        w = int(rng.integers(0, 3))
        lo, hi = min(0, dn) - w, max(0, dn) + w
        expect = brute.brute_banded_global(q, s, sig, 5, 2, lo, hi)
        assert oracle.score_banded(q, s, sig, 5, 2, lo, hi) == expect


def test_band_ub_is_an_upper_bound():
    # every alignment visiting diagonal d scores <= UB(d)
    rng = np.random.default_rng(41)
    sig = synth.dna_matrix(2, -3)
    for _ in range(25):
        m, n = rng.integers(1, 6, size=2)
        q, s = _dna(rng, m), _dna(rng, n)
        al = brute.alignments(m, n)
        sc = brute.global_scores(q, s, sig, 5, 2)
        for d in range(-m, n + 1):
            ub = oracle.band_ub(m, n, 2, 5, 2, d)
            for k, ops in enumerate(al):
                i = j = 0
                visits = d == 0
                for op in ops:
                    i += op in "MD"
                    j += op in "MI"
                    visits |= (j - i) == d
                if visits:
                    assert sc[k] <= ub


def test_band_doubling_is_exact():
    b = synth.long_dna_pairs(npairs=12, lmin=60, lmax=200, seed=8)
    for p in range(b.npairs):
        q = b.q_codes[b.q_off[p]:b.q_off[p + 1]]
        t = b.t_codes[b.t_off[p]:b.t_off[p + 1]]
        full = oracle.score(q, t, b.matrix, 5, 2, "global")
        for w0 in (0, 1, 4, 16):
            sc, w, tries = oracle.banded_doubling(q, t, b.matrix, 5, 2, w0)
            assert sc == full
            assert w >= w0
        wmin = oracle.min_certified_w(q, t, b.matrix, 5, 2)
        sc, w, _ = oracle.banded_doubling(q, t, b.matrix, 5, 2, wmin)
        assert w == wmin and sc == full
        if wmin > 0:
            # one below the minimum does not certify: doubling must move on
            sc2, w2, tries2 = oracle.banded_doubling(q, t, b.matrix, 5, 2, wmin - 1)
            assert tries2 >= 1 and sc2 == full


def _in_block_region(i, j, m, lo, hi, K):
    # the band [lo, hi] rounded out to blocks of K columns (written from the
    # definition independently of the C predicate)
    if j == 0:
        return -i >= lo
    b = (j - 1) // K
    first = max(1, b * K + 1 - hi)
    last = min(m, b * K + K - lo)
    if i == 0:
        return first == 1
    return first <= i <= last


def _brute_region(q, s, sig, alpha, beta, member):
    al = brute.alignments(len(q), len(s))
    sc = brute.global_scores(q, s, sig, alpha, beta)
    best = None
    for k, ops in enumerate(al):
        i = j = 0
        ok = member(0, 0)
        for op in ops:
            i += op in "MD"
            j += op in "MI"
            ok = ok and member(i, j)
        if ok:
            best = int(sc[k]) if best is None else max(best, int(sc[k]))
    return best


def test_block_region_vs_path_restricted_brute():
    rng = np.random.default_rng(43)
    sig = synth.dna_matrix(2, -3)
    for _ in range(60):
        m, n = rng.integers(1, 6, size=2)
        q, s = _dna(rng, m), _dna(rng, n)
        dn = n - m
        w = int(rng.integers(0, 3))
        lo, hi = min(0, dn) - w, max(0, dn) + w
        K = int(rng.integers(1, 4))
        want = _brute_region(q, s, sig, 5, 2, lambda i, j: _in_block_region(i, j, m, lo, hi, K))
        assert oracle.score_blockband(q, s, sig, 5, 2, lo, hi, K) == want


def test_block_region_contains_band_and_certifies_no_later():
    b = synth.long_dna_pairs(npairs=10, lmin=80, lmax=250, seed=12)
    for p in range(b.npairs):
        q = b.q_codes[b.q_off[p]:b.q_off[p + 1]]
        t = b.t_codes[b.t_off[p]:b.t_off[p + 1]]
        m, n = len(q), len(t)
        full = oracle.score(q, t, b.matrix, 5, 2, "global")
        for w in (0, 3, 10):
            lo, hi = min(0, n - m) - w, max(0, n - m) + w
            strict = oracle.score_banded(q, t, b.matrix, 5, 2, lo, hi)
            block = oracle.score_blockband(q, t, b.matrix, 5, 2, lo, hi, 16)
            assert strict <= block <= full
        assert oracle.score_blockband(q, t, b.matrix, 5, 2, -m, n, 16) == full
        for w0 in (0, 4, 32):
            sc, w_used, _ = oracle.banded_doubling_blocks(q, t, b.matrix, 5, 2, w0, 16)
            sc2, w_strict, _ = oracle.banded_doubling(q, t, b.matrix, 5, 2, w0)
            assert sc == full == sc2
            assert w0 <= w_used <= max(w_strict, w0)
