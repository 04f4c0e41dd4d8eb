"""GPU parity of batch plans (include/gotoh_plan.h): preallocated runs, CUDA
graph replay and autotuned launch configurations all give the oracle's
scores bit for bit; capacity violations are reported per pair on the
device, never read out of bounds."""
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


def _dev(*arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _oracle(qc, qo, tc, to, mat, a, b, mode):
    out, errs = oracle.batch(qc, qo, tc, to, mat, a, b, mode, nthreads=NTHREADS)
    return out, errs


def assert_same(got, want, what=""):
    got = np.asarray(got, dtype=np.int64)
    want = np.asarray(want, dtype=np.int64)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} mismatches, first {bad[:8]} got {got[bad[:8]]} want {want[bad[:8]]}"


def _mixed(seed, n=700, lmax=700, alphabet=4):
    """Lengths from 0 to lmax: every tile width, ragged tails, pairs wider
    than the widest tile (intra-sequence kernel), empty sequences."""
    rng = np.random.default_rng(seed)
    lq = rng.integers(0, lmax + 1, size=n)
    lt = np.clip(lq + rng.integers(-40, 41, size=n), 0, None)
    lq[:4] = [0, 0, 5, 513]
    lt[:4] = [0, 7, 0, 520]
    freqs = None if alphabet == 4 else np.concatenate([synth.PROTEIN_BACKGROUND, np.zeros(4)])
    qc, qo = synth.random_sequences(rng, lq, alphabet, freqs)
    tc, to = synth.random_sequences(rng, lt, alphabet, freqs)
    return qc, qo, tc, to


@pytest.mark.parametrize("mode", MODES)
def test_plan_run_matches_oracle(mode):
    qc, qo, tc, to = _mixed(101)
    mat = synth.dna_matrix(2, -3)
    want, _ = _oracle(qc, qo, tc, to, mat, 5, 2, mode)
    with ga.Plan(mat, 5, 2, mode, max_pairs=1000, max_residues=max(qo[-1], to[-1]), max_len=1024) as plan:
        d = _dev(qc, qo, tc, to)
        for _ in range(2):  # the workspace is reused: a second run starts clean
            got = plan.run(*d)
            st = plan.stats()
            assert_same(got.cpu().numpy(), want, f"plan {mode}")
            assert st["status"] == 0
            assert st["cells"] == int(np.sum(np.diff(qo) * np.diff(to)))


@pytest.mark.parametrize("tiles16,tiles32,conc", [(0x1ff, 0x1ff, 1), (0x155, 0x1ff, 0), (0x100, 0x100, 1),
                                                   (0x013, 0x0, 0), (0x0, 0x0, 1)])
def test_plan_tunings_are_exact(tiles16, tiles32, conc):
    # any set of bin tiles (pairs wider than every active tile fall back to
    # the intra-sequence kernel), bins in order or concurrent
    qc, qo, tc, to = _mixed(102, n=400, lmax=600)
    mat = synth.dna_matrix(2, -3)
    d = _dev(qc, qo, tc, to)
    for mode in MODES:
        want, _ = _oracle(qc, qo, tc, to, mat, 5, 2, mode)
        with ga.Plan(mat, 5, 2, mode, 400, max(qo[-1], to[-1]), 700) as plan:
            plan.tuning = ga.Tuning(tiles16, tiles32, conc, 0)
            got = plan.run(*d)
            assert_same(got.cpu().numpy(), want, f"tuning {tiles16:#x}/{tiles32:#x}/{conc} {mode}")
            assert plan.stats()["status"] == 0


@pytest.mark.parametrize("lanes_alt", [ga.TILE_ALT_MASK, 0x0007F, 0x1D400, 0x00055])
def test_plan_alternative_lane_groups_are_exact(lanes_alt):
    # packed tiles with 8 lanes x 2K columns (narrow tiles) or 32 lanes x
    # K/2 columns (wide tiles) instead of 16 lanes x K: pairs of every width
    # up to 600 columns, every mode, bins in order and concurrent
    qc, qo, tc, to = _mixed(103, n=700, lmax=600)
    mat = synth.dna_matrix(2, -3)
    d = _dev(qc, qo, tc, to)
    for mode in MODES:
        want, _ = _oracle(qc, qo, tc, to, mat, 5, 2, mode)
        with ga.Plan(mat, 5, 2, mode, 700, max(qo[-1], to[-1]), 700) as plan:
            for conc in (0, 1):
                plan.tuning = ga.Tuning((1 << 17) - 1, (1 << 17) - 1, conc, lanes_alt)
                got = plan.run(*d)
                assert_same(got.cpu().numpy(), want, f"lanes_alt {lanes_alt:#x} {conc} {mode}")
                assert plan.stats()["status"] == 0


def test_plan_rejects_lane_groups_without_an_alternative():
    with ga.Plan(synth.dna_matrix(2, -3), 5, 2, "global", 10, 1000, 100) as plan:
        with pytest.raises(ga.GotohError):
            plan.tuning = ga.Tuning((1 << 17) - 1, 0, 1, 1 << 8)  # tile 8 (K = 14) has none


def test_plan_graph_replay_reads_new_inputs():
    # capture once, then overwrite the captured input buffers with another
    # batch of the same pair count and replay: the replay scores that batch
    mat = synth.dna_matrix(2, -3)
    n, cap = 600, 600 * 320
    batches = [synth.mutated_dna_pairs(npairs=n, seed=synth.SEED_BASE + 77 + k) for k in range(3)]
    q = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    t = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    qo = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    to = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    scores = torch.empty(n, dtype=torch.int32, device="cuda")

    def load(b):
        q[:len(b.q_codes)] = torch.from_numpy(b.q_codes).cuda()
        t[:len(b.t_codes)] = torch.from_numpy(b.t_codes).cuda()
        qo.copy_(torch.from_numpy(b.q_off))
        to.copy_(torch.from_numpy(b.t_off))

    for mode in ("global", "semiglobal", "local"):
        with ga.Plan(mat, 5, 2, mode, n, cap, 400) as plan:
            plan.tuning = ga.Tuning((1 << 17) - 1, (1 << 17) - 1, 1, 0)
            load(batches[0])
            torch.cuda.synchronize()
            plan.capture(q, qo, t, to, scores)
            for b in batches:
                load(b)
                plan.launch()
                st = plan.stats()
                want, _ = _oracle(b.q_codes, b.q_off, b.t_codes, b.t_off, mat, 5, 2, mode)
                assert_same(scores.cpu().numpy(), want, f"replay {mode}")
                assert st["status"] == 0


def test_plan_protein_runs_on_the_profile_kernel():
    qc, qo, tc, to = _mixed(103, n=120, lmax=400, alphabet=24)
    mat = synth.blosum62()
    d = _dev(qc, qo, tc, to)
    for mode in MODES:
        want, _ = _oracle(qc, qo, tc, to, mat, 11, 1, mode)
        with ga.Plan(mat, 11, 1, mode, 120, max(qo[-1], to[-1]), 600) as plan:
            got = plan.run(*d)
            assert_same(got.cpu().numpy(), want, f"protein plan {mode}")
        with ga.Plan(mat, 11, 1, mode, 120, max(qo[-1], to[-1]), 600) as plan:
            got = torch.empty(120, dtype=torch.int32, device="cuda")
            plan.capture(*d, got)
            plan.launch()
            assert_same(got.cpu().numpy(), want, f"protein graph {mode}")


def test_plan_capacity_and_residue_errors():
    # a sequence longer than max_len, one ending beyond max_residues and one
    # with a residue outside the alphabet: those pairs are INT32_MIN with a
    # device status, every other pair exact
    rng = np.random.default_rng(104)
    lq = rng.integers(1, 200, size=64)
    lt = rng.integers(1, 100, size=64)
    lq[10] = 300   # > max_len
    qc, qo = synth.random_sequences(rng, lq, 4)
    tc, to = synth.random_sequences(rng, lt, 4)
    qc[qo[20]] = 9  # residue >= alphabet size
    mat = synth.dna_matrix(2, -3)
    cap = int(qo[-1]) - 3  # the last query ends beyond the capacity
    want, _ = _oracle(qc, qo, tc, to, mat, 5, 2, "global")
    d = _dev(qc, qo, tc, to)
    with ga.Plan(mat, 5, 2, "global", 64, max(cap, int(to[-1])), 256) as plan:
        got = plan.run(*d).cpu().numpy()
        st = plan.stats()
    bad = {10, 20, 63}
    assert all(got[i] == INT32_MIN for i in bad)
    keep = [i for i in range(64) if i not in bad]
    assert_same(got[keep], want[keep], "capacity")
    assert st["status"] in (5, 7)  # GA_ERR_RESIDUE or GA_ERR_RANGE, whichever came first


def test_plan_arguments_checked_synchronously():
    mat = synth.dna_matrix(2, -3)
    with ga.Plan(mat, 5, 2, "global", 10, 1000, 100) as plan:
        d = _dev(*synth.random_sequences(np.random.default_rng(1), [5] * 11, 4),
                 *synth.random_sequences(np.random.default_rng(2), [5] * 11, 4))
        with pytest.raises(ga.GotohError) as e:
            plan.run(*d)  # 11 pairs > max_pairs
        assert e.value.code == 1
        with pytest.raises(ga.GotohError) as e:
            plan.launch()  # nothing captured
        assert e.value.code == 1
    with pytest.raises(ga.GotohError):
        ga.Plan(mat, 5, 2, "global", 0, 1000, 100)


def test_plan_autotune_keeps_scores_exact():
    b = synth.mutated_dna_pairs(npairs=20_000, seed=synth.SEED_BASE + 91)
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    for mode in ("global", "local"):
        with ga.Plan(b.matrix, b.alpha, b.beta, mode, b.npairs, max(b.q_off[-1], b.t_off[-1]), 400) as plan:
            tuning, ms = plan.autotune(*d, reps=3)
            assert ms > 0 and tuning["tiles16"] is not None
            got = plan.run(*d)
            want, _ = _oracle(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta, mode)
            assert_same(got.cpu().numpy(), want, f"autotuned {mode}")


def test_plan_run_enqueues_without_blocking_the_host():
    # a run enqueues kernels only: queued behind ~0.1 s of device work on its
    # stream (a bounded busy-wait of a fixed cycle count), it returns while
    # that work is still running, and the scores, read after the stream is
    # synchronised, equal the oracle's
    b = synth.mutated_dna_pairs(npairs=5000, seed=synth.SEED_BASE + 93)
    d = _dev(b.q_codes, b.q_off, b.t_codes, b.t_off)
    want, _ = _oracle(b.q_codes, b.q_off, b.t_codes, b.t_off, b.matrix, b.alpha, b.beta, "global")
    s = torch.cuda.Stream()
    with ga.Plan(b.matrix, b.alpha, b.beta, "global", b.npairs, max(b.q_off[-1], b.t_off[-1]), 400) as plan:
        plan.run(*d, stream=s)  # first run: lazy module loading, workspace touched
        s.synchronize()
        scores = torch.empty(b.npairs, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(s):
            torch.cuda._sleep(200_000_000)
        plan.run(*d, scores=scores, stream=s)
        still_busy = not s.query()
        s.synchronize()
        assert still_busy, "plan.run waited for the stream"
        assert_same(scores.cpu().numpy(), want, "async plan run")
        assert plan.stats(stream=s)["status"] == 0
