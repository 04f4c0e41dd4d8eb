"""GPU parity at the full benchmark sizes, in the launch configuration the
bench times: the whole workload runs on the GPU in one call (the serving
stream in one submission).  Every output is compared with the CPU oracle:
the 1M-pair batch against the oracle run here; the 20k long pairs (full DP,
band doubling and the learned band) and the 200k serving requests against
the oracle's scores stored in tests/golden/ by make_fullsize_goldens.py
(which calls only oracle/ and synth/; each file carries a digest of the
generated inputs, checked first).  The protein search, 1e8 pairs, is compared
on every query against 4,096 sampled targets (the 64 longest included).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.golden import make_fullsize_goldens as goldens

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_07610_gb300 as ga  # noqa: E402

NTHREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _built():
    ga.build()
    ga.load()


def _dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _sample(rng, sizes, k, longest):
    """k random indices plus the `longest` largest by `sizes`."""
    top = np.argsort(sizes)[-longest:]
    pick = rng.choice(len(sizes), size=k, replace=False)
    return np.unique(np.concatenate([pick, top]))


def test_config2_full_batch():
    # 1M mutated DNA pairs, global and semi-global, as one bench step (one
    # multi-mode call): every score of both modes against the oracle
    # (8.7e10 cells, about 20 s on 16 cores)
    b = synth.mutated_dna_pairs(npairs=1_000_000, seed=synth.SEED_BASE + 2)
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    modes = ("global", "semiglobal")
    got, st = ga.align_batch_modes(*d, b.matrix, b.alpha, b.beta, modes, stats=True)
    assert st["status"] == 0 and st["pairs"] == 2 * b.npairs and st["pairs_int16"] == 2 * b.npairs
    assert st["cells"] == 2 * b.cells()
    got = got.cpu().numpy().astype(np.int64)
    for k, mode in enumerate(modes):
        want, errs = oracle.batch(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta,
                                  mode, nthreads=NTHREADS)
        assert not errs.any()
        np.testing.assert_array_equal(got[k], want)


def test_config3_full_database_sampled():
    # 512 protein queries x 200k targets, local, BLOSUM62 11/1: the whole
    # search on the packed query-profile kernel, every query against 4,096
    # sampled targets that include the 64 longest (4.6e11 cells, about 2 min
    # on 16 cores)
    cr = synth.protein_database()
    d = _dev(cr.q_codes, cr.q_off, cr.t_codes, cr.t_off)
    got, st = ga.align_cross(*d, cr.matrix, cr.alpha, cr.beta, "local", stats=True)
    assert st["status"] == 0
    tl = np.diff(cr.t_off)
    tsel = _sample(np.random.default_rng(3), tl, 4096 - 64, 64)
    ts = [cr.t_codes[cr.t_off[i]:cr.t_off[i + 1]] for i in tsel]
    tc, to = synth.pack_csr(ts)
    want, errs = oracle.cross(cr.q_codes, cr.q_off, tc, to, cr.matrix, cr.alpha, cr.beta, "local",
                              nthreads=NTHREADS)
    assert not errs.any()
    np.testing.assert_array_equal(got.cpu().numpy()[:, tsel].astype(np.int64), want)


def _golden(path, digest):
    g = np.load(path)
    assert str(g["digest"]) == digest, f"{os.path.basename(path)}: the generated inputs changed; " \
        "rerun tests/golden/make_fullsize_goldens.py"
    return g["scores"].astype(np.int64)


def test_config4_full_dp_band_and_learned_band_full():
    # 20k long DNA pairs, global: full DP, band doubling from the default
    # start and from the learned start (a predictor trained here on 1,000
    # other pairs): every score of all three against the oracle
    from paper_2205_07610_gb300 import band
    b = synth.long_dna_pairs(npairs=20_000)
    want = _golden(goldens.LONG_PATH, goldens.long_digest(b))
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    full, st = ga.align_batch(*d, b.matrix, b.alpha, b.beta, "global", stats=True)
    assert st["status"] == 0
    np.testing.assert_array_equal(full.cpu().numpy().astype(np.int64), want)
    banded, w_used = ga.align_banded(*d, b.matrix, b.alpha, b.beta, default_w0=16)
    np.testing.assert_array_equal(banded.cpu().numpy().astype(np.int64), want)
    assert int(w_used.min()) >= 0
    tr = synth.long_dna_pairs(npairs=1000, seed=synth.SEED_BASE + 400)
    pred, _ = band.train(*_dev(tr.q_codes, tr.q_off, tr.t_codes, tr.t_off), b.matrix, b.alpha, b.beta,
                         synth.mlp_init(synth.SEED_BASE + 401),
                         synth.minibatches(tr.npairs, 128, 300, synth.SEED_BASE + 402), lr=2e-3)
    learned, _, st = pred.align(*d, b.matrix, b.alpha, b.beta, stats=True)
    assert st["status"] == 0
    np.testing.assert_array_equal(learned.cpu().numpy().astype(np.int64), want)


def test_config5_full_serving_stream():
    # the whole 200k-request serving stream submitted to the server at once
    # (mixed DNA / protein, local / global, lengths up to 50k): every result
    # against the oracle
    s = synth.serving_stream()
    want = _golden(goldens.SERVING_PATH, goldens.serving_digest(s))
    cells = np.diff(s.q_off) * np.diff(s.t_off)
    with ga.Server(arena_bytes=32 << 30, max_inflight=65536, max_tasks=1 << 22) as srv:
        d = srv.add_scoring(*s.dna_scoring)
        p = srv.add_scoring(*s.protein_scoring)
        sid = np.where(s.protein, p, d).astype(np.int32)
        first = srv.submit(s.q_codes, s.q_off, s.t_codes, s.t_off, s.mode, sid)
        srv.drain(600_000)
        res = srv.poll(s.nreq + 16)
    assert len(res) == s.nreq
    res = res[np.argsort(res["id"])]
    assert np.array_equal(res["id"], first + np.arange(s.nreq))
    assert np.all(res["status"] == 0)
    assert np.array_equal(res["cells"], cells)
    np.testing.assert_array_equal(res["score"].astype(np.int64), want)
