"""GPU parity of ga_align_banded (global mode, certified band doubling).

Every score must equal the full-DP oracle score, and the band at which the GPU
accepts must be exactly the oracle's: the oracle runs the same doubling on
the same block-rounded region (band [lo, hi] rounded out to 16-column blocks),
so every intermediate region score and certificate decision has to agree for
w_used to match.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_07610_gb300 as ga  # noqa: E402

BLOCK = 16
NTHREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _built():
    ga.build()
    ga.load()


def _run(b, w0=None, default_w0=16):
    d = "cuda"
    q = torch.from_numpy(np.ascontiguousarray(b.q_codes)).to(d)
    qo = torch.from_numpy(np.ascontiguousarray(b.q_off)).to(d)
    t = torch.from_numpy(np.ascontiguousarray(b.t_codes)).to(d)
    to = torch.from_numpy(np.ascontiguousarray(b.t_off)).to(d)
    w0t = None if w0 is None else torch.from_numpy(np.asarray(w0, dtype=np.int32)).to(d)
    sc, wu, st = ga.align_banded(q, qo, t, to, b.matrix, b.alpha, b.beta, w0=w0t,
                                 default_w0=default_w0, stats=True)
    torch.cuda.synchronize()
    return sc.cpu().numpy().astype(np.int64), wu.cpu().numpy(), st


def _check(b, w0s):
    got, wu, st = _run(b, w0=w0s)
    full, errs = oracle.batch(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta,
                              "global", nthreads=NTHREADS)
    bad = np.nonzero(got != full)[0]
    assert len(bad) == 0, f"{len(bad)} score mismatches, e.g. {bad[:5]} {got[bad[:5]]} {full[bad[:5]]}"
    for p in range(b.npairs):
        q = b.q_codes[b.q_off[p]:b.q_off[p + 1]]
        t = b.t_codes[b.t_off[p]:b.t_off[p + 1]]
        sc, w_used, _ = oracle.banded_doubling_blocks(q, t, b.matrix, b.alpha, b.beta, int(w0s[p]),
                                                      BLOCK)
        assert sc == full[p]
        assert wu[p] == w_used, (p, len(q), len(t), int(w0s[p]), int(wu[p]), w_used)
    assert st["status"] == 0
    return st


def test_banded_short_pairs_many_w0():
    rng = np.random.default_rng(3)
    b = synth.long_dna_pairs(npairs=300, lmin=20, lmax=700, seed=55)
    w0s = rng.choice([0, 1, 3, 8, 20, 64, 400], size=b.npairs)
    st = _check(b, w0s)
    assert st["band_retries"] > 0 and st["banded_cells"] > 0


def test_banded_long_pairs():
    b = synth.long_dna_pairs(npairs=24, lmin=1000, lmax=4000, seed=synth.SEED_BASE + 4)
    rng = np.random.default_rng(9)
    w0s = rng.choice([0, 16, 128, 1024], size=b.npairs)
    st = _check(b, w0s)
    assert st["banded_cells"] < st["cells"]


def test_banded_skewed_and_edge_pairs():
    rng = np.random.default_rng(11)
    lq = [1, 5, 600, 40, 3000, 700, 1, 0, 17, 900]
    lt = [900, 1, 30, 2000, 2500, 700, 1, 5, 0, 1800]
    qc, qo = synth.random_sequences(rng, lq)
    tc, to = synth.random_sequences(rng, lt)
    for (ma, mi), al, be in (((2, -3), 5, 2), ((1, -1), 1, 1)):
        b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(ma, mi), al, be, "skew")
        _check(b, rng.integers(0, 40, size=b.npairs))


def test_banded_protein_falls_back_to_full_dp():
    cr = synth.protein_database(nq=1, qmin=200, qmax=300, nt=30, median=250, seed=7)
    q = [cr.q_codes[cr.q_off[0]:cr.q_off[1]]] * cr.nt
    t = [cr.t_codes[cr.t_off[k]:cr.t_off[k + 1]] for k in range(cr.nt)]
    qc, qo = synth.pack_csr(q)
    tc, to = synth.pack_csr(t)
    b = synth.Batch(qc, qo, tc, to, cr.matrix, 11, 1, "protein")
    got, wu, _ = _run(b)
    full, _ = oracle.batch(qc, qo, tc, to, cr.matrix, 11, 1, "global", nthreads=NTHREADS)
    assert np.array_equal(got, full)
    assert (wu == -1).all()


def test_banded_packed_and_int32_kernels():
    # sigma_max + alpha <= 24 runs on the packed int16x2 kernel, larger on the
    # int32 kernel; both must accept at the oracle's width with its score
    b = synth.long_dna_pairs(npairs=40, lmin=300, lmax=3000, seed=57)
    w0s = np.random.default_rng(12).choice([0, 4, 32, 256], size=b.npairs)
    for al, be in ((5, 2), (22, 2), (23, 2), (40, 3)):
        _check(synth.Batch(b.q_codes, b.q_off, b.t_codes, b.t_off, synth.dna_matrix(2, -3), al, be, "k"), w0s)


def test_banded_single_diagonal_and_super_stage_edges():
    # equal lengths with w0 = 0 (a band of one diagonal), widths around the
    # 512 / 1,024 columns of one packed super-stage, and several super-stages
    rng = np.random.default_rng(13)
    lens = [100, 511, 512, 513, 1023, 1024, 1025, 2600]
    qs, ts = [], []
    for L in lens:
        q = rng.integers(0, 4, size=L).astype(np.uint8)
        qs += [q, q]
        ts += [q.copy(), rng.integers(0, 4, size=L).astype(np.uint8)]
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "diag")
    st = _check(b, np.zeros(b.npairs, dtype=np.int64))
    assert st["band_retries"] > 0


def test_banded_schedule_spacing_boundaries():
    # The packed band kernel starts super-stage s (64 blocks of 16 columns)
    # D * s iterations after super-stage 0, D = max(128, min(m, B - 1008) + 1)
    # for a window of B = 2w + |n - m| + 16 rows: shapes at the 128 floor
    # and just above it, D clipped by a short query, a query much longer
    # than its target, and widths around multiples of 1,024 columns; each as
    # a related pair (a mutated copy) and an unrelated one.
    rng = np.random.default_rng(17)
    shapes = [(1500, 1500, 559), (1500, 1500, 560), (1500, 1500, 561), (3000, 3300, 400),
              (300, 4000, 0), (130, 5000, 0), (100, 5000, 0), (5000, 100, 0),
              (2047, 2047, 16), (2048, 2048, 16), (2049, 2049, 16), (4097, 4097, 100)]
    qs, ts, w0s = [], [], []
    for m, n, w in shapes:
        q = rng.integers(0, 4, size=m).astype(np.uint8)
        t = q.copy()
        if n <= m:
            t = t[:n]
        else:
            t = np.concatenate([t, rng.integers(0, 4, size=n - m).astype(np.uint8)])
        sub = rng.random(n) < 0.05
        t[sub] = (t[sub] + rng.integers(1, 4, size=int(sub.sum()))) % 4
        qs += [q, q]
        ts += [t, rng.integers(0, 4, size=n).astype(np.uint8)]
        w0s += [w, w]
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "spacing")
    st = _check(b, np.asarray(w0s, dtype=np.int64))
    assert st["band_retries"] > 0
