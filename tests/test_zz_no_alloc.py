"""ga_align_long_noalloc against ga_align_long, through the C ABI.

The no-allocation entry point exists for callers that cannot allocate device
memory while they align (device memory held by a pooling allocator, or a
latency-critical loop that cannot take cudaMalloc's implicit synchronisation).
Its scratch lives in one file-scope device array shared by every call, so
this test makes two calls in a row with different pairs and checks that each
gives exactly the score of the allocating entry point (integer scores: the
tolerance is zero).  It runs alone in a fresh process or after every other
test (pytest collects this file last).
"""
import ctypes

import numpy as np
import pytest

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


def _call_noalloc(lib, q, t, matrix, go, ge, mode):
    sc, keep = ga.make_scoring(matrix, go, ge)
    out = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
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


def test_noalloc_matches_long_on_two_calls_in_a_row(lib):
    rng = np.random.default_rng(2024)
    dna = synth.dna_matrix(2, -3)
    cases = [
        # (m, n, alphabet, matrix, gap open, gap extend, mode)
        (3000, 2500, 4, dna, 5, 2, 1),                   # DNA, global
        (1400, 1700, 20, synth.blosum62(), 11, 1, 0),    # protein, local
        (900, 4100, 4, dna, 5, 2, 2),                    # DNA, semi-global
    ]
    for m, n, alph, mat, go, ge, mode in cases:
        q = torch.from_numpy(rng.integers(0, alph, size=m).astype(np.uint8)).cuda()
        t = torch.from_numpy(rng.integers(0, alph, size=n).astype(np.uint8)).cuda()
        rc1, got = _call_noalloc(lib, q, t, mat, go, ge, mode)
        rc2, want = _call_long(lib, q, t, mat, go, ge, mode)
        assert rc1 == 0 and rc2 == 0
        assert got == want, (m, n, mode)


def test_noalloc_rejects_sequences_beyond_its_limit(lib):
    big = torch.zeros(ga.NOALLOC_MAX_LEN + 1, dtype=torch.uint8, device="cuda")
    small = torch.zeros(10, dtype=torch.uint8, device="cuda")
    rc, _ = _call_noalloc(lib, big, small, synth.dna_matrix(2, -3), 5, 2, 1)
    assert rc == 1  # GA_ERR_ARG, nothing enqueued
