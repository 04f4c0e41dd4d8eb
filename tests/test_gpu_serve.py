"""GPU tests of the strip-task kernel: long pairs on many warps
(ga_align_long) and the alignment server (continuous batching).

Every score is compared bit for bit with the CPU oracle; the server test also
checks that each request's result is the same when it runs alone and when it
runs in the mix of a Poisson stream.
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
MODES = ("local", "global", "semiglobal")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ga.build()
    ga.load()


def _long_cases(rng):
    """(q, t) pairs around the strip width and with either orientation."""
    cases = []
    for m, n in ((1, 1), (0, 700), (700, 0), (5, 512), (512, 513), (513, 512), (1500, 1025),
                 (300, 4100), (4100, 300), (2048, 2048)):
        q = rng.integers(0, 4, size=m).astype(np.uint8)
        if n >= 40 and m >= 40:
            qc, qo = synth.pack_csr([q])
            tc, to = synth.mutate(rng, qc, qo, np.array([0.1]), np.array([0.3]))
            t = tc[to[0]:to[1]].astype(np.uint8)[:n]
            if len(t) < n:
                t = np.concatenate([t, rng.integers(0, 4, size=n - len(t)).astype(np.uint8)])
        else:
            t = rng.integers(0, 4, size=n).astype(np.uint8)
        cases.append((q, t))
    return cases


@pytest.mark.parametrize("mode", MODES)
def test_long_pairs_on_strip_warps(mode):
    rng = np.random.default_rng(21)
    for (ma, mi), al, be in (((2, -3), 5, 2), ((1, -1), 1, 1)):
        mat = synth.dna_matrix(ma, mi)
        for q, t in _long_cases(rng):
            got, st = ga.align_long(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), mat, al,
                                    be, mode, stats=True)
            ref = oracle.score(q, t, mat, al, be, mode)
            assert int(got.item()) == ref, (mode, len(q), len(t), int(got.item()), ref)
            assert st["status"] == 0


def test_long_protein_pairs_on_strip_warps():
    rng = np.random.default_rng(22)
    mat = synth.blosum62()
    bg = np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    for m, n in ((800, 1700), (2600, 600), (1, 33)):
        q = rng.choice(24, size=m, p=bg).astype(np.uint8)
        t = rng.choice(24, size=n, p=bg).astype(np.uint8)
        for mode in MODES:
            got = ga.align_long(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), mat, 11, 1, mode)
            assert int(got.item()) == oracle.score(q, t, mat, 11, 1, mode), (m, n, mode)


def _stream(nreq, lmax, seed):
    s = synth.serving_stream(nreq=nreq, lmax=lmax, seed=seed)
    return s


def _oracle_scores(s):
    ref = np.zeros(s.nreq, dtype=np.int64)
    for prot in (0, 1):
        for md in (0, 1):
            idx = np.nonzero((s.protein == prot) & (s.mode == md))[0]
            if not len(idx):
                continue
            mat, al, be = s.protein_scoring if prot else s.dna_scoring
            qs = [s.q_codes[s.q_off[i]:s.q_off[i + 1]] for i in idx]
            ts = [s.t_codes[s.t_off[i]:s.t_off[i + 1]] for i in idx]
            qc, qo = synth.pack_csr(qs)
            tc, to = synth.pack_csr(ts)
            r, _ = oracle.batch(qc, qo, tc, to, mat, al, be, "global" if md else "local",
                                nthreads=NTHREADS)
            ref[idx] = r
    return ref


def _serve(srv, s, ids_dna, ids_prot, idx=None, release=True):
    idx = np.arange(s.nreq) if idx is None else np.asarray(idx)
    qs = [s.q_codes[s.q_off[i]:s.q_off[i + 1]] for i in idx]
    ts = [s.t_codes[s.t_off[i]:s.t_off[i + 1]] for i in idx]
    qc, qo = synth.pack_csr(qs)
    tc, to = synth.pack_csr(ts)
    sid = np.where(s.protein[idx] == 1, ids_prot, ids_dna).astype(np.int32)
    rel = None
    if release:
        t0 = srv.clock_ns() + 2_000_000
        rel = (t0 + (s.arrival[idx] - s.arrival[idx][0]) * 1e9).astype(np.int64)
    first = srv.submit(qc, qo, tc, to, s.mode[idx].astype(np.int32), sid, rel)
    srv.drain(120_000)
    res = srv.poll(len(idx) + 16)
    assert len(res) == len(idx)
    order = np.argsort(res["id"])
    res = res[order]
    assert np.array_equal(res["id"], first + np.arange(len(idx)))
    return res


def test_server_mixed_stream_alone_and_in_mix():
    s = _stream(600, 6000, 77)
    ref = _oracle_scores(s)
    with ga.Server(arena_bytes=256 << 20, max_inflight=1024, max_tasks=1 << 16) as srv:
        d = srv.add_scoring(*s.dna_scoring)
        p = srv.add_scoring(*s.protein_scoring)
        mix = _serve(srv, s, d, p)
        assert np.all(mix["status"] == 0)
        np.testing.assert_array_equal(mix["score"], ref)
        assert np.all(mix["release_ns"] <= mix["admit_ns"]) and np.all(mix["admit_ns"] <= mix["done_ns"])
        assert np.array_equal(mix["cells"], np.diff(s.q_off) * np.diff(s.t_off))
        # the same requests one at a time
        pick = np.random.default_rng(3).choice(s.nreq, size=40, replace=False)
        for i in pick:
            alone = _serve(srv, s, d, p, idx=[i], release=False)
            assert alone["score"][0] == mix["score"][i] == ref[i]
        st = srv.stats()
        assert st["completed"] == s.nreq + len(pick) and st["kernel_launches"] >= 1


def test_server_admits_by_device_memory():
    # an arena that holds the largest request (a 20000 x 20000 pair needs
    # 6.2 MB of strip edges) but far less than the stream: requests wait for
    # memory, all finish exactly
    s = _stream(200, 20000, 78)
    ref = _oracle_scores(s)
    arena = 8 << 20
    with ga.Server(arena_bytes=arena, max_inflight=64, max_tasks=4096) as srv:
        d = srv.add_scoring(*s.dna_scoring)
        p = srv.add_scoring(*s.protein_scoring)
        res = _serve(srv, s, d, p, release=False)
        np.testing.assert_array_equal(res["score"], ref)
        assert srv.stats()["arena_high_water"] <= arena


def test_server_rejects_bad_requests():
    with ga.Server(arena_bytes=16 << 20) as srv:
        d = srv.add_scoring(synth.dna_matrix(2, -3), 5, 2)
        q = np.zeros(ga.SERVE_MAX_LEN + 1, dtype=np.uint8)
        with pytest.raises(ga.GotohError):
            srv.submit(q, [0, len(q)], q[:10], [0, 10], [0], [d])
        with pytest.raises(ga.GotohError):
            srv.submit(q[:10], [0, 10], q[:10], [0, 10], [0], [d + 5])
        with pytest.raises(ga.GotohError):
            srv.submit(q[:10], [0, 10], q[:10], [0, 10], [3], [d])
        big = np.zeros(40000, dtype=np.uint8)  # 78 strip edges of 40001 rows: 25 MB > 16 MB arena
        with pytest.raises(ga.GotohError):
            srv.submit(big, [0, 40000], big, [0, 40000], [1], [d])
        # a residue outside the alphabet is reported per request
        bad = np.full(20, 7, dtype=np.uint8)
        srv.submit(bad, [0, 20], q[:10], [0, 10], [1], [d])
        srv.drain(30_000)
        r = srv.poll()
        assert len(r) == 1 and r["status"][0] == 5  # GA_ERR_RESIDUE


def test_bounded_wait_runs_out_and_reports():
    # failure detection without a GPU fault: the strip kernel's edge wait,
    # run alone on a device flag that nothing writes, gives up after its
    # limit and reports GA_ERR_TIMEOUT; a satisfied flag returns at once, and
    # the context stays usable (an alignment afterwards is exact)
    status, waited = ga.probe_bounded_wait(0, 1, 2_000_000)
    assert status == 6  # GA_ERR_TIMEOUT
    assert 2_000_000 <= waited < 500_000_000
    status, waited = ga.probe_bounded_wait(7, 7, 2_000_000)
    assert status == 0 and waited < 2_000_000
    rng = np.random.default_rng(77)
    q = rng.integers(0, 4, size=900).astype(np.uint8)
    t = rng.integers(0, 4, size=1100).astype(np.uint8)
    mat = synth.dna_matrix(2, -3)
    got = ga.align_long(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), mat, 5, 2, "global")
    assert int(got.item()) == oracle.score(q, t, mat, 5, 2, "global")
