"""GPU parity of the packed int16x2 long-pair kernel (pairs whose shorter
sequence exceeds the 512 columns of the widest inter-sequence tile, alphabets
of <= 4 symbols) against the CPU oracle, bit for bit.

The kernel stores every cell relative to a per-lane base, so the cases aim
at what that representation must survive: scores far outside int16 (long
identical and long unrelated pairs), many renormalisations (rows in the
thousands), one and several super-stages of 1,024 columns with ragged last
halves (a last super-stage whose right half is all padding), both
orientations, every mode, and the largest scoring the kernel accepts
(sigma_max + alpha = 128) next to the smallest it hands to the int32 kernel.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    ga.build()
    ga.load()


def _run(b, mode):
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.q_codes, b.q_off, b.t_codes, b.t_off)]
    got, st = ga.align_batch(*d, b.matrix, b.alpha, b.beta, mode, stats=True)
    want, errs = oracle.batch(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta, mode,
                              nthreads=NTHREADS)
    assert not errs.any()
    got = got.cpu().numpy().astype(np.int64)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{mode}: {len(bad)} mismatches, pairs {bad[:6]} got {got[bad[:6]]} want {want[bad[:6]]}"
    return want, st


@pytest.mark.parametrize("mode", MODES)
def test_packed_long_widths_and_orientation(mode):
    rng = np.random.default_rng(91)
    # shorter sides around the super-stage (1,024) and half (512) boundaries
    cols = [513, 600, 1000, 1023, 1024, 1025, 1536, 2047, 2049, 3100]
    lq, lt = [], []
    for k, c in enumerate(cols):
        r = int(rng.integers(c, 6000))
        lq.append(r if k % 2 else c)   # both orientations
        lt.append(c if k % 2 else r)
    qc, qo = synth.random_sequences(rng, np.array(lq))
    tc, to = synth.random_sequences(rng, np.array(lt))
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "packed-long")
    _, st = _run(b, mode)
    assert st["status"] == 0 and st["pairs_int16"] == len(cols)


@pytest.mark.parametrize("mode", MODES)
def test_packed_long_scores_beyond_int16(mode):
    rng = np.random.default_rng(92)
    same = rng.integers(0, 4, size=20_000).astype(np.uint8)
    a_run = np.zeros(20_000, np.uint8)          # AAAA...
    c_run = np.ones(6000, np.uint8)             # CCCC...
    mutated = synth.long_dna_pairs(npairs=6, lmin=8000, lmax=16000, seed=93)
    qs = [same, a_run, c_run] + [mutated.q_codes[mutated.q_off[p]:mutated.q_off[p + 1]] for p in range(6)]
    ts = [same.copy(), c_run, a_run] + [mutated.t_codes[mutated.t_off[p]:mutated.t_off[p + 1]] for p in range(6)]
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    b = synth.Batch(qc, qo, tc, to, synth.dna_matrix(2, -3), 5, 2, "beyond-int16")
    want, st = _run(b, mode)
    assert want[0] == 40_000                      # 20,000 matches in every mode
    if mode == "global":  # 6,000 mismatches and a gap of 14,000
        assert want[1] == want[2] == -3 * 6000 - (5 + 2 * 13_999)
    assert st["pairs_int16"] == len(qs) and st["pairs_int32_rerun"] == 0


@pytest.mark.parametrize("mode", MODES)
def test_packed_long_scoring_limit(mode):
    # sigma_max + alpha = 128 runs packed; 129 runs on the int32 kernel
    lb = synth.long_dna_pairs(npairs=10, lmin=600, lmax=4000, seed=94)
    for alpha, packed in ((125, True), (126, False)):
        b = synth.Batch(lb.q_codes, lb.q_off, lb.t_codes, lb.t_off, synth.dna_matrix(3, -3), alpha, 1,
                        f"limit-{alpha}")
        _, st = _run(b, mode)
        assert (st["pairs_int16"], st["pairs_int32"]) == ((10, 0) if packed else (0, 10)), (alpha, st)
    # a linear gap (alpha = beta) and an asymmetric 4 x 4 matrix
    rng = np.random.default_rng(95)
    mat = rng.integers(-6, 7, size=(4, 4)).astype(np.int8)
    for alpha, beta in ((4, 4), (9, 3)):
        b = synth.Batch(lb.q_codes, lb.q_off, lb.t_codes, lb.t_off, mat, alpha, beta, "asym")
        _run(b, mode)
