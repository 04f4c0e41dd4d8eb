"""GPU parity at the full benchmark sizes, in the launch configuration the
bench times: the whole workload runs on the GPU in one call (the serving
stream in one submission).  The 1M-pair batch is compared with the CPU
oracle pair by pair in full; for the larger workloads a seeded sample of the
outputs (the longest pairs, targets and requests included) is, with every
query of the protein search against 4,096 targets.  Properties that hold at
any size (banded scores equal full-DP scores) are checked on every pair.
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


def test_config4_full_dp_and_band_sampled():
    # 20k long DNA pairs, global: full DP on every pair, band doubling from
    # the default start; every banded score equals the full-DP score, and a
    # sample of 150 pairs plus the 4 largest equals the oracle
    b = synth.long_dna_pairs(npairs=20_000)
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    full, st = ga.align_batch(*d, b.matrix, b.alpha, b.beta, "global", stats=True)
    assert st["status"] == 0
    band, w_used = ga.align_banded(*d, b.matrix, b.alpha, b.beta, default_w0=16)
    assert torch.equal(band, full)
    assert int(w_used.min()) >= 0
    m, n = b.lengths()
    idx = _sample(np.random.default_rng(4), m * n, 150, 4)
    sub = b.subset(idx)
    want, errs = oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, b.matrix, b.alpha, b.beta,
                              "global", nthreads=NTHREADS)
    assert not errs.any()
    np.testing.assert_array_equal(full.cpu().numpy()[idx].astype(np.int64), want)


def test_config5_full_serving_stream_sampled():
    # the whole 200k-request serving stream submitted to the server at once
    # (mixed DNA / protein, local / global, lengths up to 50k); a sample of
    # 2,000 results plus the 3 largest requests equals the oracle
    s = synth.serving_stream()
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
    idx = _sample(np.random.default_rng(5), cells, 2000, 3)
    for prot in (False, True):  # the oracle on the sample, by scoring and mode
        for md in (0, 1):
            sel = idx[(s.protein[idx] == prot) & (s.mode[idx] == md)]
            if not len(sel):
                continue
            mat, al, be = s.protein_scoring if prot else s.dna_scoring
            qc, qo = synth.pack_csr([s.q_codes[s.q_off[i]:s.q_off[i + 1]] for i in sel])
            tc, to = synth.pack_csr([s.t_codes[s.t_off[i]:s.t_off[i + 1]] for i in sel])
            want, errs = oracle.batch(qc, qo, tc, to, mat, al, be, "global" if md else "local",
                                      nthreads=NTHREADS)
            assert not errs.any()
            np.testing.assert_array_equal(res["score"][sel].astype(np.int64), want)
