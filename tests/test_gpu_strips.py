"""GPU parity of the strip kernel's packed cells (ga_align_long and the
server run the same strips) against the CPU oracle, bit for bit.

A strip is two 256-column halves in the int16 halves of every register, each
value relative to a per-lane base: the cases aim at scores far outside int16
(long identical protein pairs in local mode, long unrelated pairs in global
mode), lengths around the 256 / 512-column half and strip boundaries, both
orientations, every mode, and the scoring limit of the packed strips
(sigma_max + alpha = 128 packed, 129 on the int32 strips).
"""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    ga.build()
    ga.load()


def _long(q, t, mat, al, be, mode):
    return ga.align_long(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), mat, al, be, mode).item()


@pytest.mark.parametrize("mode", MODES)
def test_strip_boundaries_both_orientations(mode):
    rng = np.random.default_rng(61)
    dna = synth.dna_matrix(2, -3)
    for m, n in ((300, 255), (300, 256), (300, 257), (700, 511), (700, 512), (700, 513),
                 (2000, 1023), (513, 3000), (64, 5000), (4100, 900)):
        q = rng.integers(0, 4, size=m).astype(np.uint8)
        t = rng.integers(0, 4, size=n).astype(np.uint8)
        assert _long(q, t, dna, 5, 2, mode) == oracle.score(q, t, dna, 5, 2, mode), (m, n, mode)


@pytest.mark.parametrize("mode", MODES)
def test_strip_scores_beyond_int16(mode):
    rng = np.random.default_rng(62)
    b62 = synth.blosum62()
    bg = np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    prot = rng.choice(24, size=9000, p=bg).astype(np.uint8)
    # an 85 %-identity copy: the local score is far above 32767
    qc, qo = synth.pack_csr([prot])
    tc, to = synth.mutate(rng, qc, qo, 0.15, 0.1, 24, bg)
    got = _long(prot, tc[to[0]:to[1]].astype(np.uint8), b62, 11, 1, mode)
    want = oracle.score(prot, tc[to[0]:to[1]], b62, 11, 1, mode)
    assert got == want
    if mode == "local":
        assert want > 32767
    dna = synth.dna_matrix(2, -3)
    a_run, c_run = np.zeros(20_000, np.uint8), np.ones(6000, np.uint8)
    got = _long(a_run, c_run, dna, 5, 2, mode)
    assert got == oracle.score(a_run, c_run, dna, 5, 2, mode)
    if mode == "global":
        assert got < -32768


@pytest.mark.parametrize("mode", MODES)
def test_strip_scoring_limit(mode):
    rng = np.random.default_rng(63)
    q = rng.integers(0, 4, size=3000).astype(np.uint8)
    qc, qo = synth.pack_csr([q])
    tc, to = synth.mutate(rng, qc, qo, 0.1, 0.3)
    t = tc[to[0]:to[1]].astype(np.uint8)
    mat = synth.dna_matrix(3, -3)
    for alpha in (125, 126):  # sigma_max + alpha = 128 (packed) and 129 (int32 strips)
        assert _long(q, t, mat, alpha, 1, mode) == oracle.score(q, t, mat, alpha, 1, mode), (alpha, mode)


@pytest.mark.parametrize("mode", MODES)
def test_strip_rows_around_batch_boundaries(mode):
    # the strip loop runs batches of 32 rows, the interior ones without
    # per-row checks once every lane is past its first rows (iteration 64)
    # and before row R: row counts around those boundaries, one and several
    # strips, both orientations
    rng = np.random.default_rng(64)
    dna = synth.dna_matrix(2, -3)
    b62 = synth.blosum62()
    for R in (1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 97, 98, 127, 128, 129, 130, 160, 161, 191, 192, 193, 225):
        for C in (R, 300, 1200):
            q = rng.integers(0, 4, size=R).astype(np.uint8)
            t = rng.integers(0, 4, size=C).astype(np.uint8)
            assert _long(q, t, dna, 5, 2, mode) == oracle.score(q, t, dna, 5, 2, mode), (R, C, mode)
            assert _long(t, q, dna, 5, 2, mode) == oracle.score(t, q, dna, 5, 2, mode), (C, R, mode)
        pq = rng.integers(0, 20, size=R).astype(np.uint8)
        pt = rng.integers(0, 20, size=700).astype(np.uint8)
        assert _long(pq, pt, b62, 11, 1, mode) == oracle.score(pq, pt, b62, 11, 1, mode), (R, "protein", mode)
