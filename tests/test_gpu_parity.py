"""GPU parity: every score of the CUDA path equals the CPU oracle bit for bit.

Inputs are seeded synthetic workloads (synth/); the oracle (oracle/) and the
CUDA library share nothing but those inputs.  Cases span several lane tiles,
every inter-sequence bin edge, ragged tails, swapped orientation, the long
multi-stage kernel, protein (profile path), int16 overflow with the exact int32
rerun, statically int32 pairs, empty sequences and device-detected errors.
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

MODES = ["local", "global", "semiglobal"]
NTHREADS = max(1, min(32, os.cpu_count() or 1))
INT32_MIN = -(2 ** 31)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ga.build()
    ga.load()


def _dev(b):
    d = "cuda"
    return (torch.from_numpy(np.ascontiguousarray(b.q_codes)).to(d),
            torch.from_numpy(np.ascontiguousarray(b.q_off)).to(d),
            torch.from_numpy(np.ascontiguousarray(b.t_codes)).to(d),
            torch.from_numpy(np.ascontiguousarray(b.t_off)).to(d))


def gpu_batch(b, mode, stats=False):
    q, qo, t, to = _dev(b)
    r = ga.align_batch(q, qo, t, to, b.matrix, b.alpha, b.beta, mode, stats=stats)
    torch.cuda.synchronize()
    if stats:
        return r[0].cpu().numpy(), r[1]
    return r.cpu().numpy()


def oracle_batch(b, mode):
    out, errs = oracle.batch(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta,
                             mode, nthreads=NTHREADS)
    assert not errs.any()
    return out


def assert_same(got, want, what=""):
    got = np.asarray(got, dtype=np.int64)
    want = np.asarray(want, dtype=np.int64)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} mismatches, first {bad[:8]} got {got[bad[:8]]} want {want[bad[:8]]}"


def _pairs(rng, lens_q, lens_t, alphabet=4, freqs=None):
    qc, qo = synth.random_sequences(rng, lens_q, alphabet, freqs)
    tc, to = synth.random_sequences(rng, lens_t, alphabet, freqs)
    return qc, qo, tc, to


@pytest.mark.parametrize("mode", MODES)
def test_config1_uniform_150(mode):
    b = synth.uniform_dna_pairs()  # 1,000 pairs of 150 x 150, +2/-3, 5/2
    got, st = gpu_batch(b, mode, stats=True)
    assert_same(got, oracle_batch(b, mode), f"config1 {mode}")
    assert st["status"] == 0
    assert st["cells"] == b.cells()
    assert st["pairs_int16"] == b.npairs


@pytest.mark.parametrize("mode", MODES)
def test_mixed_lengths_all_bins(mode):
    """Lengths 1..700 with both orientations: every bin, ragged tails, long pairs."""
    rng = np.random.default_rng(101)
    n = 2500
    lq = rng.integers(1, 700, size=n)
    lt = np.clip(lq + rng.integers(-60, 60, size=n), 1, None)
    swap = rng.random(n) < 0.3
    lt[swap] = rng.integers(1, 700, size=int(swap.sum()))
    qc, qo, tc, to = _pairs(rng, lq, lt)
    # cheap gaps make paths through the row-0 / column-0 borders optimal often
    for (ma, mi), al, be in (((2, -3), 5, 2), ((2, -3), 1, 1), ((1, -4), 2, 1)):
        b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(ma, mi), al, be, "mixed")
        got = gpu_batch(b, mode)
        assert_same(got, oracle_batch(b, mode), f"mixed {mode} {ma}/{mi} {al}/{be}")


@pytest.mark.parametrize("mode", ["global", "semiglobal"])
def test_config2_subset(mode):
    b = synth.mutated_dna_pairs(npairs=20000, seed=synth.SEED_BASE + 2)
    got, st = gpu_batch(b, mode, stats=True)
    assert_same(got, oracle_batch(b, mode), f"config2 subset {mode}")
    assert st["pairs_int16"] == b.npairs and st["pairs_int32_rerun"] == 0


@pytest.mark.parametrize("mode", MODES)
def test_bin_edges_and_small(mode):
    rng = np.random.default_rng(7)
    # every tile width (16 lanes x K columns: 96 .. 320 in steps of 16, 384,
    # 512) and its neighbours, short pairs and a pair past the widest tile
    edges = [1, 2, 3, 15, 16, 17, 31, 32, 33] + [w + d for w in range(96, 321, 16) for d in (-1, 0, 1)] + \
            [383, 384, 385, 511, 512, 513, 600]
    lq, lt = [], []
    for e in edges:
        for other in (1, e, e + 7, max(1, e - 9), 300):
            lq.append(e); lt.append(other)
            lq.append(other); lt.append(e)
    qc, qo, tc, to = _pairs(rng, lq, lt)
    for (ma, mi), al, be in (((2, -3), 5, 2), ((1, -1), 2, 1), ((3, -1), 3, 3)):
        b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(ma, mi), al, be, "edges")
        assert_same(gpu_batch(b, mode), oracle_batch(b, mode), f"edges {mode} {ma}/{mi} {al}/{be}")


@pytest.mark.parametrize("mode", MODES)
def test_empty_and_identical(mode):
    seqs = [np.zeros(0, np.uint8), synth.encode("A"), synth.encode("ACGT" * 40),
            synth.encode("GATTACA" * 30)]
    q, t = [], []
    for a in seqs:
        for c in seqs:
            q.append(a); t.append(c)
    qc, qo = synth.pack_csr(q)
    tc, to = synth.pack_csr(t)
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "empty")
    assert_same(gpu_batch(b, mode), oracle_batch(b, mode), f"empty/identical {mode}")


def test_asymmetric_dna_matrix_swapped_orientation():
    rng = np.random.default_rng(9)
    mat = rng.integers(-4, 5, size=(4, 4)).astype(np.int8)
    lq = rng.integers(5, 400, size=600)
    lt = rng.integers(5, 400, size=600)
    qc, qo, tc, to = _pairs(rng, lq, lt)
    b = synth.Batch(qc, qo, tc, to, mat, 4, 1, "asym")
    for mode in MODES:
        assert_same(gpu_batch(b, mode), oracle_batch(b, mode), f"asymmetric {mode}")


def test_local_int16_overflow_rerun_is_exact():
    """Match score 100: identical pairs of length >= 327 exceed int16; they are
    detected on the device and recomputed exactly in int32."""
    rng = np.random.default_rng(5)
    seqs = [rng.integers(0, 4, size=L).astype(np.uint8) for L in (100, 300, 330, 400, 500, 512)]
    q = seqs + [s.copy() for s in seqs]
    t = seqs + [rng.integers(0, 4, size=len(s)).astype(np.uint8) for s in seqs]
    qc, qo = synth.pack_csr(q)
    tc, to = synth.pack_csr(t)
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(100, -90), 120, 60, "overflow")
    got, st = gpu_batch(b, "local", stats=True)
    want = oracle_batch(b, "local")
    assert_same(got, want, "local overflow rerun")
    assert want.max() > 32767
    assert st["pairs_int32_rerun"] >= 3


@pytest.mark.parametrize("mode", ["global", "semiglobal"])
def test_statically_int32_pairs(mode):
    rng = np.random.default_rng(13)
    lq = rng.integers(50, 500, size=300)
    lt = rng.integers(50, 500, size=300)
    qc, qo, tc, to = _pairs(rng, lq, lt)
    for al, be in ((500, 100), (1000, 800)):
        b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), al, be, "int32")
        got, st = gpu_batch(b, mode, stats=True)
        assert_same(got, oracle_batch(b, mode), f"int32 {mode} {al}/{be}")
        assert st["pairs_int32"] > 0


@pytest.mark.parametrize("mode", MODES)
def test_long_pairs_multistage(mode):
    rng = np.random.default_rng(17)
    lq = [520, 1000, 3000, 1500, 2048, 4100]
    lt = [600, 1300, 2500, 3500, 2048, 700]
    qc, qo, tc, to = _pairs(rng, lq, lt)
    for (ma, mi), al, be in (((2, -3), 5, 2), ((2, -3), 1, 1)):
        b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(ma, mi), al, be, "long")
        assert_same(gpu_batch(b, mode), oracle_batch(b, mode), f"long {mode} {al}/{be}")
    lb = synth.long_dna_pairs(npairs=8, lmin=1000, lmax=5000, seed=21)
    assert_same(gpu_batch(lb, mode), oracle_batch(lb, mode), f"long mutated {mode}")


@pytest.mark.parametrize("mode", MODES)
def test_protein_blosum62(mode):
    rng = np.random.default_rng(19)
    bg = np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    lq = rng.integers(1, 700, size=300)
    lt = rng.integers(1, 700, size=300)
    qc, qo, tc, to = _pairs(rng, lq, lt, 24, bg)
    for al, be in ((11, 1), (2, 1)):
        b = synth.Batch(qc, qo, tc, to, synth.blosum62(), al, be, "protein")
        assert_same(gpu_batch(b, mode), oracle_batch(b, mode), f"protein {mode} {al}/{be}")


def test_device_detected_errors():
    rng = np.random.default_rng(23)
    qc, qo, tc, to = _pairs(rng, [10, 20, 30], [10, 20, 30])
    qc = qc.copy()
    qc[15] = 7  # residue code outside A..T in pair 1
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "bad")
    got, st = gpu_batch(b, "global", stats=True)
    assert st["status"] == 5  # GA_ERR_RESIDUE
    assert got[1] == INT32_MIN
    good = synth.Batch(*_pairs(np.random.default_rng(23), [10, 20, 30], [10, 20, 30]),
                       synth.dna_matrix(2, -3), 5, 2)
    want = oracle_batch(good, "global")
    assert got[0] == want[0] and got[2] == want[2]
    # decreasing offsets: the bad pair is flagged, the others are exact
    qo2 = qo.copy()
    qo2[2] = qo2[1] - 3
    b2 = synth.Batch(qc, qo2, tc, to, synth.dna_matrix(2, -3), 5, 2, "badoff")
    got2, st2 = gpu_batch(b2, "global", stats=True)
    assert st2["status"] in (1, 5) and got2[1] == INT32_MIN


def test_host_entry_point_matches_device():
    b = synth.mutated_dna_pairs(npairs=3000, seed=77)
    for mode in MODES:
        host = ga.align_batch_host(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha,
                                   b.beta, mode)
        assert_same(host, gpu_batch(b, mode), f"host {mode}")


def test_host_entry_point_in_chunks():
    # more pairs than one copy chunk (2^18): chunks start at arbitrary residue
    # offsets (not multiples of 16), each is packed from its own first residue
    rng = np.random.default_rng(5)
    n = 700_000
    qc, qo = synth.random_sequences(rng, rng.integers(1, 40, size=n))
    tc, to = synth.random_sequences(rng, rng.integers(1, 40, size=n))
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "chunks")
    for mode in MODES:
        host, st = ga.align_batch_host(qc, qo, tc, to, b.matrix, 5, 2, mode, stats=True)
        assert_same(host, gpu_batch(b, mode), f"host chunks {mode}")
        assert st["pairs"] == n and st["status"] == 0
    sub = rng.choice(n, size=300, replace=False)
    want, _ = oracle.batch(*_subset(b, sub), b.matrix, 5, 2, "global", nthreads=NTHREADS)
    host = ga.align_batch_host(qc, qo, tc, to, b.matrix, 5, 2, "global")
    assert_same(host[sub], want, "host chunks vs oracle")


def test_batch_modes_entry_point():
    # several modes from one packing of the inputs: every row equals the
    # single-mode entry point, mixed lengths (inter-sequence bins, long pairs,
    # empty sequences) included; bad modes are rejected before any work
    qc, qo, tc, to = _pairs(np.random.default_rng(8), np.random.default_rng(9).integers(0, 700, size=900),
                            np.random.default_rng(10).integers(0, 700, size=900))
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "modes")
    q, qo_d, t, to_d = _dev(b)
    modes = ["semiglobal", "local", "global", "local"]
    got, st = ga.align_batch_modes(q, qo_d, t, to_d, b.matrix, 5, 2, modes, stats=True)
    assert tuple(got.shape) == (4, b.npairs) and st["status"] == 0 and st["pairs"] == 4 * b.npairs
    for k, mode in enumerate(modes):
        assert_same(got[k].cpu().numpy(), oracle_batch(b, mode), f"modes row {k} {mode}")
    with pytest.raises(ga.GotohError) as e:
        ga.align_batch_modes(q, qo_d, t, to_d, b.matrix, 5, 2, [1, 5])
    assert e.value.code == 1


def test_batch_modes_overflow_errors_and_empty():
    # one multi-mode call whose two local plans both queue int16 overflows
    # for the int32 rerun, with empty sequences, long-class pairs and one
    # invalid residue: every row equals the single-mode entry point
    # (INT32_MIN for the invalid pair, status GA_ERR_RESIDUE), the valid
    # pairs equal the oracle, and the host entry point gives the same rows
    rng = np.random.default_rng(15)
    lq = list(rng.integers(0, 520, size=300)) + [0, 5, 0, 513, 600]
    lt = list(rng.integers(0, 520, size=300)) + [7, 0, 0, 600, 513]
    qs = [rng.integers(0, 4, size=int(n)).astype(np.uint8) for n in lq]
    ts = [rng.integers(0, 4, size=int(n)).astype(np.uint8) for n in lt]
    for i, L in enumerate((330, 400, 480, 510)):  # identical: local score 100 L > 32767
        qs[10 + i] = rng.integers(0, 4, size=L).astype(np.uint8)
        ts[10 + i] = qs[10 + i].copy()
    qs[40] = qs[40].copy()
    qs[40][len(qs[40]) // 2] = 7  # outside the 4-symbol alphabet
    assert len(qs[40]) > 0
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(100, -90), 120, 60, "modes-errors")
    q, qo_d, t, to_d = _dev(b)
    modes = ["local", "global", "local", "semiglobal"]
    got, st = ga.align_batch_modes(q, qo_d, t, to_d, b.matrix, 120, 60, modes, stats=True)
    got = got.cpu().numpy()
    assert st["status"] == 5 and st["pairs_int32_rerun"] >= 8
    valid = np.ones(b.npairs, dtype=bool)
    valid[40] = False
    for k, mode in enumerate(modes):
        assert_same(got[k], gpu_batch(b, mode), f"modes row {k} {mode} vs single mode")
        assert got[k][40] == INT32_MIN
        want, errs = oracle.batch(*_subset(b, np.nonzero(valid)[0]), b.matrix, 120, 60, mode, nthreads=NTHREADS)
        assert not errs.any()
        assert_same(got[k][valid], want, f"modes row {k} {mode} vs oracle")
    assert oracle_batch_local_max(b, valid) > 32767
    host, hst = ga.align_batch_host_modes(qc, qo, tc, to, b.matrix, 120, 60, modes, stats=True)
    assert hst["status"] == 5
    assert_same(host.ravel(), got.ravel(), "host modes vs device modes")


def oracle_batch_local_max(b, valid):
    want, _ = oracle.batch(*_subset(b, np.nonzero(valid)[0]), b.matrix, b.alpha, b.beta, "local",
                           nthreads=NTHREADS)
    return int(want.max())


def test_host_modes_entry_point():
    # several modes of the same pairs from one host copy, over several copy
    # chunks; every row equals the device entry point in its mode, and the
    # global row a sample of the oracle
    rng = np.random.default_rng(6)
    n = 600_000
    qc, qo = synth.random_sequences(rng, rng.integers(0, 60, size=n))
    tc, to = synth.random_sequences(rng, rng.integers(0, 60, size=n))
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "modes")
    modes = ["global", "semiglobal", "local", "global"]
    host, st = ga.align_batch_host_modes(qc, qo, tc, to, b.matrix, 5, 2, modes, stats=True)
    assert host.shape == (4, n) and st["status"] == 0 and st["pairs"] == 4 * n
    for k, mode in enumerate(modes):
        assert_same(host[k], gpu_batch(b, mode), f"host modes row {k} {mode}")
    sub = rng.choice(n, size=300, replace=False)
    want, _ = oracle.batch(*_subset(b, sub), b.matrix, 5, 2, "local", nthreads=NTHREADS)
    assert_same(host[2][sub], want, "host modes local vs oracle")
    with pytest.raises(ga.GotohError) as e:
        ga.align_batch_host_modes(qc[:10], qo[:3], tc[:10], to[:3], b.matrix, 5, 2, [0, 3])
    assert e.value.code == 1


def _subset(b, idx):
    qs = [b.q_codes[b.q_off[i]:b.q_off[i + 1]] for i in idx]
    ts = [b.t_codes[b.t_off[i]:b.t_off[i + 1]] for i in idx]
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    return qc, qo, tc, to


def test_protein_cross_local_bins_and_stages():
    # queries in every column bin of the packed protein kernel (<= 128, 256,
    # 320, 384, 448, 512 columns), both sides of each bin edge, and longer
    # ones that run in stages; queries of a bin are paired by length, so some
    # pairs mix stage counts and odd bins leave a half without a query;
    # targets from empty to long, one with an invalid residue
    rng = np.random.default_rng(12)
    bg = np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    qlens = [0, 1, 50, 128, 129, 256, 257, 300, 320, 321, 384, 385, 448, 449, 512, 513, 700, 1100]
    tlens = list(rng.integers(1, 900, size=150)) + [0, 1, 2, 2000]
    qs = [rng.choice(24, size=n, p=bg).astype(np.uint8) for n in qlens]
    ts = [rng.choice(24, size=int(n), p=bg).astype(np.uint8) for n in tlens]
    ts[5] = qs[11][100:600].copy()  # a strong local hit
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    mat = synth.blosum62()
    d = "cuda"
    dev = [torch.from_numpy(a).to(d) for a in (qc, qo, tc, to)]
    got, st = ga.align_cross(*dev, mat, 11, 1, "local", stats=True)
    want, _ = oracle.cross(qc, qo, tc, to, mat, 11, 1, "local", nthreads=NTHREADS)
    assert_same(got.cpu().numpy().ravel(), want.ravel(), "protein cross local")
    assert st["status"] == 0
    # an invalid residue in one target: that column is INT32_MIN, the rest exact
    tc2 = tc.copy()
    tc2[to[7]] = 30
    got2, st2 = ga.align_cross(dev[0], dev[1], torch.from_numpy(tc2).to(d), dev[3], mat, 11, 1, "local",
                               stats=True)
    g2 = got2.cpu().numpy()
    assert st2["status"] == 5 and np.all(g2[:, 7] == np.iinfo(np.int32).min)
    keep = [l for l in range(len(ts)) if l != 7]
    assert_same(g2[:, keep].ravel(), want[:, keep].ravel(), "protein cross, invalid target")


def test_protein_cross_int16_rerun():
    # identical 7000-residue sequences: the local score exceeds the int16 range,
    # the pair is flagged and recomputed exactly in int32
    rng = np.random.default_rng(13)
    bg = np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    q = rng.choice(24, size=7000, p=bg).astype(np.uint8)
    qs = [q, q[:300]]
    ts = [q.copy(), rng.choice(24, size=500, p=bg).astype(np.uint8)]
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    mat = synth.blosum62()
    dev = [torch.from_numpy(a).cuda() for a in (qc, qo, tc, to)]
    got, st = ga.align_cross(*dev, mat, 11, 1, "local", stats=True)
    want, _ = oracle.cross(qc, qo, tc, to, mat, 11, 1, "local", nthreads=NTHREADS)
    assert want[0, 0] > 32767
    assert_same(got.cpu().numpy().ravel(), want.ravel(), "protein rerun")
    assert st["pairs_int32_rerun"] >= 1


def test_protein_cross_packed5_positions():
    # the targets reach the kernel packed 5 bits each, six residues per word:
    # targets of every length 1..41 (and 82 more) start at every position
    # mod 6, the set
    # starts 7 residues into its buffer (a chunk of a larger set), and every
    # code of the 24-symbol alphabet appears; the queries span two tiles
    rng = np.random.default_rng(29)
    lens = np.concatenate([np.arange(1, 42), rng.integers(1, 42, size=82)])
    ts = [rng.integers(0, 24, size=L).astype(np.uint8) for L in lens]
    tc, to = synth.pack_csr(ts)
    pre = rng.integers(0, 24, size=7).astype(np.uint8)
    tc2 = np.concatenate([pre, tc])
    to2 = to + 7
    qs = [rng.integers(0, 24, size=L).astype(np.uint8) for L in (90, 150, 300, 700)]
    qc, qo = synth.pack_csr(qs)
    mat = synth.blosum62()
    dev = [torch.from_numpy(a).cuda() for a in (qc, qo, tc2, to2)]
    got, st = ga.align_cross(*dev, mat, 11, 1, "local", stats=True)
    assert st["status"] == 0
    assert sorted({int(o) % 6 for o in to2[:-1]}) == list(range(6))
    want, _ = oracle.cross(qc, qo, tc, to, mat, 11, 1, "local", nthreads=NTHREADS)
    assert_same(got.cpu().numpy().ravel(), want.ravel(), "packed5 targets")


def test_protein_cross_rerun_list_overflow():
    # more flagged pairs than one rerun list holds (65,536): 260 identical
    # queries against 260 identical targets (sigma = 127 on the diagonal, so
    # every such local score is 300 x 127 = 38,100 > 32,767) plus 40 random
    # targets; the flagged pairs beyond the list are found again from their
    # marks and recomputed in int32, the others keep their int16 scores
    rng = np.random.default_rng(17)
    mat = rng.integers(-4, 5, size=(24, 24)).astype(np.int8)
    np.fill_diagonal(mat, 127)
    same = rng.integers(0, 24, size=300).astype(np.uint8)
    qc, qo = synth.pack_csr([same] * 260)
    tc, to = synth.pack_csr([same] * 260 + [rng.integers(0, 24, size=300).astype(np.uint8) for _ in range(40)])
    dev = [torch.from_numpy(a).cuda() for a in (qc, qo, tc, to)]
    got, st = ga.align_cross(*dev, mat, 11, 1, "local", stats=True)
    got = got.cpu().numpy().astype(np.int64)
    assert st["status"] == 0 and st["pairs_int32_rerun"] == 260 * 260
    assert oracle.score(same, same, mat, 11, 1, "local") == 38100
    assert np.all(got[:, :260] == 38100)
    rc, ro = synth.pack_csr([tc[to[k]:to[k + 1]] for k in range(260, 300)])
    want, _ = oracle.cross(qc[:300], qo[:2], rc, ro, mat, 11, 1, "local", nthreads=NTHREADS)
    assert_same(got[:, 260:].ravel(), np.tile(want, (260, 1)).ravel(), "non-flagged pairs")


@pytest.mark.parametrize("mode", MODES)
def test_cross_small(mode):
    cr = synth.protein_database(nq=6, qmin=20, qmax=300, nt=80, median=120, seed=31)
    d = "cuda"
    q = torch.from_numpy(cr.q_codes).to(d); qo = torch.from_numpy(cr.q_off).to(d)
    t = torch.from_numpy(cr.t_codes).to(d); to = torch.from_numpy(cr.t_off).to(d)
    got = ga.align_cross(q, qo, t, to, cr.matrix, cr.alpha, cr.beta, mode).cpu().numpy()
    want, errs = oracle.cross(cr.q_codes, cr.q_off, cr.t_codes, cr.t_off, cr.matrix, cr.alpha,
                              cr.beta, mode, nthreads=NTHREADS)
    assert_same(got.ravel(), want.ravel(), f"cross protein {mode}")
    # DNA cross
    rng = np.random.default_rng(3)
    qc, qo_ = synth.random_sequences(rng, rng.integers(10, 300, size=5))
    tc, to_ = synth.random_sequences(rng, rng.integers(10, 300, size=40))
    got = ga.align_cross(torch.from_numpy(qc).to(d), torch.from_numpy(qo_).to(d),
                         torch.from_numpy(tc).to(d), torch.from_numpy(to_).to(d),
                         synth.dna_matrix(2, -3), 5, 2, mode).cpu().numpy()
    want, _ = oracle.cross(qc, qo_, tc, to_, synth.dna_matrix(2, -3), 5, 2, mode, nthreads=NTHREADS)
    assert_same(got.ravel(), want.ravel(), f"cross dna {mode}")


@pytest.mark.parametrize("mode", MODES)
def test_long_entry_point(mode):
    rng = np.random.default_rng(41)
    for (m, n, prot) in ((5000, 4200, False), (1300, 1800, True), (1, 900, False)):
        A = 24 if prot else 4
        q = rng.integers(0, 20 if prot else 4, size=m).astype(np.uint8)
        t = rng.integers(0, 20 if prot else 4, size=n).astype(np.uint8)
        mat = synth.blosum62() if prot else synth.dna_matrix(2, -3)
        al, be = (11, 1) if prot else (5, 2)
        got = ga.align_long(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), mat, al, be,
                            mode).item()
        assert got == oracle.score(q, t, mat, al, be, mode), (m, n, prot, mode)


def test_protein_cross_target_rows_around_batch_boundaries():
    # the protein search runs its rows in batches of 16, the interior ones
    # without per-row checks once every lane is inside the target's rows and
    # lane 0's next edge row exists: targets of one length per call, lengths
    # around those boundaries, queries in one-stage and staged tiles
    rng = np.random.default_rng(14)
    bg = np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    qs = [rng.choice(24, size=n, p=bg).astype(np.uint8) for n in (40, 200, 448, 700)]
    qc, qo = synth.pack_csr(qs)
    mat = synth.blosum62()
    for L in (1, 2, 15, 16, 17, 18, 31, 32, 33, 34, 35, 47, 48, 49, 50, 64, 65):
        ts = [rng.choice(24, size=L, p=bg).astype(np.uint8) for _ in range(24)]
        tc, to = synth.pack_csr(ts)
        dev = [torch.from_numpy(a).cuda() for a in (qc, qo, tc, to)]
        got = ga.align_cross(*dev, mat, 11, 1, "local")
        want, _ = oracle.cross(qc, qo, tc, to, mat, 11, 1, "local", nthreads=NTHREADS)
        assert_same(got.cpu().numpy().ravel(), want.ravel(), f"protein cross, targets of {L}")
