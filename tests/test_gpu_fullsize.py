"""GPU parity at the full benchmark sizes, in the launch configuration the
bench times: the whole workload runs on the GPU in one call, and a sample of
its outputs (the longest pairs / targets included) is compared with the CPU
oracle, which computes them one by one.  Properties that hold at any size
(banded scores equal full-DP scores) are checked on every pair.
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


def test_config2_full_batch_sampled():
    # 1M mutated DNA pairs, global and semi-global, as one bench step
    b = synth.mutated_dna_pairs(npairs=1_000_000, seed=synth.SEED_BASE + 2)
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    m, n = b.lengths()
    idx = _sample(np.random.default_rng(2), m * n, 1500, 20)
    sub = b.subset(idx)
    for mode in ("global", "semiglobal"):
        got, st = ga.align_batch(*d, b.matrix, b.alpha, b.beta, mode, stats=True)
        assert st["status"] == 0 and st["pairs_int16"] == b.npairs
        assert st["cells"] == b.cells()
        want, errs = oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, b.matrix, b.alpha, b.beta,
                                  mode, nthreads=NTHREADS)
        assert not errs.any()
        np.testing.assert_array_equal(got.cpu().numpy()[idx].astype(np.int64), want)


def test_config3_full_database_sampled():
    # 512 protein queries x 200k targets, local, BLOSUM62 11/1: the whole
    # search on the packed query-profile kernel, every query against a
    # sample of targets that includes the 8 longest
    cr = synth.protein_database()
    d = _dev(cr.q_codes, cr.q_off, cr.t_codes, cr.t_off)
    got, st = ga.align_cross(*d, cr.matrix, cr.alpha, cr.beta, "local", stats=True)
    assert st["status"] == 0
    tl = np.diff(cr.t_off)
    tsel = _sample(np.random.default_rng(3), tl, 16, 8)
    ts = [cr.t_codes[cr.t_off[i]:cr.t_off[i + 1]] for i in tsel]
    tc, to = synth.pack_csr(ts)
    want, errs = oracle.cross(cr.q_codes, cr.q_off, tc, to, cr.matrix, cr.alpha, cr.beta, "local",
                              nthreads=NTHREADS)
    assert not errs.any()
    np.testing.assert_array_equal(got.cpu().numpy()[:, tsel].astype(np.int64), want)


def test_config4_full_dp_and_band_sampled():
    # 20k long DNA pairs, global: full DP on every pair, band doubling from
    # the default start; every banded score equals the full-DP score, and a
    # sample (the 4 largest pairs included) equals the oracle
    b = synth.long_dna_pairs(npairs=20_000)
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    full, st = ga.align_batch(*d, b.matrix, b.alpha, b.beta, "global", stats=True)
    assert st["status"] == 0
    band, w_used = ga.align_banded(*d, b.matrix, b.alpha, b.beta, default_w0=16)
    assert torch.equal(band, full)
    assert int(w_used.min()) >= 0
    m, n = b.lengths()
    idx = _sample(np.random.default_rng(4), m * n, 12, 4)
    sub = b.subset(idx)
    want, errs = oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, b.matrix, b.alpha, b.beta,
                              "global", nthreads=NTHREADS)
    assert not errs.any()
    np.testing.assert_array_equal(full.cpu().numpy()[idx].astype(np.int64), want)
