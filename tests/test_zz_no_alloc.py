"""ga_align_long_noalloc against ga_align_long and the CPU oracle, through the C ABI.

The no-allocation entry point exists for callers that cannot allocate device
memory while they align (device memory held by a pooling allocator, or a
latency-critical loop that cannot take cudaMalloc's implicit synchronisation).
Its scratch lives in one file-scope device array shared by every call, so
this test makes calls in a row with different pairs and checks that each
gives exactly the score of the allocating entry point and of the oracle
(integer scores: the tolerance is zero), including the paths its preparation
kernel takes alone (an empty sequence, an out-of-alphabet residue) and a
24-symbol matrix whose profile needs more than 48 KB of shared memory.  A
warm-up call comes first, as the header asks; after it, the calls leave the
device's free memory unchanged.  The file runs alone in a fresh process or
after every other test (pytest collects it last).
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_07610_gb300 as ga  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    ga.build()
    return ga.load()


def _call_noalloc(lib, q, t, matrix, go, ge, mode, out=None):
    sc, keep = ga.make_scoring(matrix, go, ge)
    if out is None:
        out = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    else:
        out.fill_(12345)
    stream = torch.cuda.current_stream()
    rc = lib.ga_align_long_noalloc(ctypes.c_void_p(q.data_ptr()), q.numel(),
                                   ctypes.c_void_p(t.data_ptr()), t.numel(), ctypes.byref(sc),
                                   mode, ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, int(out.item())


def _call_long(lib, q, t, matrix, go, ge, mode):
    sc, keep = ga.make_scoring(matrix, go, ge)
    out = torch.full((1,), 54321, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.ga_align_long(ctypes.c_void_p(q.data_ptr()), q.numel(), ctypes.c_void_p(t.data_ptr()),
                           t.numel(), ctypes.byref(sc), mode, ctypes.c_void_p(out.data_ptr()),
                           ctypes.c_void_p(stream.cuda_stream), None)
    torch.cuda.synchronize()
    return rc, int(out.item())


MODES = {0: "local", 1: "global", 2: "semiglobal"}


def test_noalloc_matches_long_and_oracle_on_calls_in_a_row(lib):
    rng = np.random.default_rng(2024)
    dna = synth.dna_matrix(2, -3)
    b62 = synth.blosum62()
    assert b62.shape == (24, 24)
    # warm-up: the first call on the device looks up (and may load) the array
    w = torch.zeros(4, dtype=torch.uint8, device="cuda")
    assert _call_noalloc(lib, w, w, dna, 5, 2, 1) == (0, 8)
    cases = [
        # (m, n, alphabet drawn, matrix, gap open, gap extend, mode)
        (3000, 2500, 4, dna, 5, 2, 1),      # DNA, global
        (1400, 1700, 20, b62, 11, 1, 0),    # protein, local (24x24 matrix: > 48 KB profile)
        (900, 4100, 4, dna, 5, 2, 2),       # DNA, semi-global
        (2100, 800, 24, b62, 11, 1, 1),     # protein incl. B Z X *, global, rows swapped
    ]
    for m, n, alph, mat, go, ge, mode in cases:
        qn = rng.integers(0, alph, size=m).astype(np.uint8)
        tn = rng.integers(0, alph, size=n).astype(np.uint8)
        q, t = torch.from_numpy(qn).cuda(), torch.from_numpy(tn).cuda()
        out = torch.empty(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc1, got = _call_noalloc(lib, q, t, mat, go, ge, mode, out)
        free1 = torch.cuda.mem_get_info()[0]
        rc2, want = _call_long(lib, q, t, mat, go, ge, mode)
        assert rc1 == 0 and rc2 == 0
        assert got == want, (m, n, mode)
        assert got == oracle.score(qn, tn, mat, go, ge, MODES[mode]), (m, n, mode)
        assert free1 == free0, "the call changed the device's free memory"


def test_noalloc_empty_sequences_and_invalid_residue(lib):
    dna = synth.dna_matrix(2, -3)
    rng = np.random.default_rng(7)
    seq = rng.integers(0, 4, size=1000).astype(np.uint8)
    dseq = torch.from_numpy(seq).cuda()
    empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
    for mode in (0, 1, 2):
        for q, t, qn, tn in ((empty, dseq, seq[:0], seq), (dseq, empty, seq, seq[:0]),
                             (empty, empty, seq[:0], seq[:0])):
            rc, got = _call_noalloc(lib, q, t, dna, 5, 2, mode)
            assert rc == 0
            assert got == oracle.score(qn, tn, dna, 5, 2, MODES[mode]), (mode, len(qn), len(tn))
    bad = seq.copy()
    bad[617] = 4  # outside the 4-symbol alphabet
    for mode in (0, 1, 2):
        rc, got = _call_noalloc(lib, torch.from_numpy(bad).cuda(), dseq, dna, 5, 2, mode)
        assert rc == 0 and got == -2**31
        # the next call on the shared array is exact again
        rc, got = _call_noalloc(lib, dseq, dseq, dna, 5, 2, mode)
        assert rc == 0 and got == oracle.score(seq, seq, dna, 5, 2, MODES[mode])


def test_noalloc_rejects_sequences_beyond_its_limit(lib):
    big = torch.zeros(ga.NOALLOC_MAX_LEN + 1, dtype=torch.uint8, device="cuda")
    small = torch.zeros(10, dtype=torch.uint8, device="cuda")
    rc, _ = _call_noalloc(lib, big, small, synth.dna_matrix(2, -3), 5, 2, 1)
    assert rc == 1  # GA_ERR_ARG, nothing enqueued
