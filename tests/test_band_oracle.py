"""Pins of the band-predictor oracles (CPU only).

* minimal certified band on block-rounded regions: a linear scan of the
  certificate predicate (not a bisection) and the doubling sequence;
* pair features: a pure-Python loop over every (sampled i, j) position pair
  comparing residues one by one, plus hand-built cases with known answers;
* the float64 network: central finite differences of the loss, closed-form
  forward passes, closed-form Adam steps and known bf16 bit patterns.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import band_features as bf
from oracle import mlp
import synth

DNA = synth.dna_matrix(2, -3)
BLOCK = 16


def _pair(rng, m, div, indel):
    q = rng.integers(0, 4, size=m).astype(np.uint8)
    qc, qo = synth.pack_csr([q])
    tc, to = synth.mutate(rng, qc, qo, np.array([div]), np.array([indel]))
    return q, tc[to[0]:to[1]].astype(np.uint8)


# ---------------------------------------------------------------- minimal band
def _certifies(q, s, w, alpha=5, beta=2):
    m, n = len(q), len(s)
    dn = n - m
    lo, hi = min(0, dn) - w, max(0, dn) + w
    sc = oracle.score_blockband(q, s, DNA, alpha, beta, lo, hi, BLOCK)
    covers = lo <= -m and hi >= n
    ub = None
    for d in (lo - 1, hi + 1):
        if -m <= d <= n:
            u = oracle.band_ub(m, n, 2, alpha, beta, d)
            ub = u if ub is None else max(ub, u)
    return covers or ub is None or sc >= ub


def test_min_certified_w_blocks_is_the_first_certifying_w():
    rng = np.random.default_rng(5)
    for trial in range(12):
        m = int(rng.integers(1, 70))
        q, s = _pair(rng, m, rng.uniform(0.0, 0.3), rng.uniform(0.1, 0.5))
        w_star = oracle.min_certified_w_blocks(q, s, DNA, 5, 2, BLOCK)
        scan = next(w for w in range(0, max(len(q), len(s)) + 1) if _certifies(q, s, w))
        assert w_star == scan, (trial, len(q), len(s))
        # the block region contains the band: it never needs a wider w
        assert w_star <= oracle.min_certified_w(q, s, DNA, 5, 2)


def test_doubling_stops_at_first_power_at_or_above_min_w():
    rng = np.random.default_rng(6)
    for _ in range(10):
        q, s = _pair(rng, int(rng.integers(20, 120)), rng.uniform(0.02, 0.3), 0.3)
        w_star = oracle.min_certified_w_blocks(q, s, DNA, 5, 2, BLOCK)
        _, w_used, _ = oracle.banded_doubling_blocks(q, s, DNA, 5, 2, 0, BLOCK)
        ladder = [0] + [1 << k for k in range(20)]
        assert w_used == next(w for w in ladder if w >= w_star)


# ---------------------------------------------------------------- features
def _brute_features(q, s):
    """The feature definition as plain loops over residues."""
    m, n, K = len(q), len(s), bf.KMER
    f = np.zeros(32, dtype=np.float32)
    f[0] = np.float32(np.log2(np.float32(1 + m))) * np.float32(0.0625)
    f[1] = np.float32(np.log2(np.float32(1 + n))) * np.float32(0.0625)
    f[2] = np.float32(np.log2(np.float32(1 + abs(n - m)))) * np.float32(0.0625)
    f[3] = np.float32(min(m, n)) / np.float32(max(m, n)) if max(m, n) else 0
    nq = max(0, m - K + 1)
    stride = max(1, math.ceil(nq / bf.MAX_SAMPLES)) if nq else 1
    sampled = list(range(0, nq, stride))
    hits = []
    for i in sampled:
        for j in range(0, max(0, n - K + 1)):
            if all(q[i + u] == s[j + u] for u in range(K)):
                hits.append((i, j))
    H = len(hits)
    matched = sorted({i for i, _ in hits})
    f[4] = np.float32(len(matched)) / np.float32(len(sampled)) if sampled else 0
    f[5] = np.float32(np.log2(np.float32(1 + H))) * np.float32(0.0625)
    for k in range(8):
        a = sum(1 for i in matched if (8 * i) // nq == k)
        b = sum(1 for i in sampled if (8 * i) // nq == k)
        f[6 + k] = np.float32(a) / np.float32(b) if b else 0
    if H:
        lo_d, hi_d = min(0, n - m), max(0, n - m)
        bins = [0] * 16
        neg = 0
        for i, j in hits:
            d = j - i
            e = d - min(max(d, lo_d), hi_d)
            bins[min(15, abs(e).bit_length())] += 1
            neg += e < 0
        for k in range(16):
            f[14 + k] = np.float32(bins[k]) / np.float32(H)
        f[30] = np.float32(neg) / np.float32(H)
    f[31] = np.float32(1.0) / np.float32(stride)
    return f


def test_features_match_brute_force_loops():
    rng = np.random.default_rng(7)
    for trial in range(14):
        m = int(rng.integers(0, 160))
        q, s = _pair(rng, m, rng.uniform(0.0, 0.2), rng.uniform(0.1, 0.5))
        if trial % 3 == 0:  # low-complexity sequences: repeated k-mers, many hits each
            q = np.tile(np.array([0, 1], dtype=np.uint8), m // 2 + 1)[:m]
            s = np.tile(np.array([0, 1], dtype=np.uint8), m // 2 + 7)[:m + 5]
        got = bf.pair_features(q, s)
        np.testing.assert_array_equal(got, _brute_features(q, s), err_msg=str(trial))


def test_features_sampling_stride():
    assert bf.sample_stride(bf.MAX_SAMPLES + bf.KMER - 1) == 1
    assert bf.sample_stride(bf.MAX_SAMPLES + bf.KMER) == 2
    assert bf.sample_stride(2 * bf.MAX_SAMPLES + bf.KMER - 1) == 2
    assert bf.sample_stride(0) == 1 and bf.sample_stride(5) == 1
    rng = np.random.default_rng(8)
    q = rng.integers(0, 4, size=5000).astype(np.uint8)
    ii, jj, qi, stride = bf.hits(q, q)
    assert stride == 3 and len(qi) == math.ceil((5000 - 11) / 3)
    assert np.all(ii == jj)                   # a random 5000-mer has no repeated 12-mer here
    assert bf.pair_features(q, q)[4] == 1.0


def test_features_hand_cases():
    acgt = np.array([0, 1, 2, 3] * 3, dtype=np.uint8)
    f = bf.pair_features(acgt, acgt)
    assert f[4] == 1 and f[5] == np.float32(1 / 16) and f[6] == 1 and f[14] == 1
    assert f[3] == 1 and f[2] == 0 and f[30] == 0 and f[31] == 1
    assert f[0] == f[1] == np.float32(np.log2(np.float32(13))) * np.float32(1 / 16)
    rng = np.random.default_rng(9)
    q = rng.integers(0, 4, size=100).astype(np.uint8)
    r = rng.integers(0, 4, size=10).astype(np.uint8)
    s = np.concatenate([r, q[:90]])          # same length, path on diagonal +10
    f = bf.pair_features(q, s)
    # every true hit has e = +10 -> bin bitlength(10) = 4; chance hits are rare
    assert f[14 + 4] > 0.9 and f[30] < 0.1
    s2 = np.concatenate([q[10:], r])         # diagonal -10
    f2 = bf.pair_features(q, s2)
    assert f2[14 + 4] > 0.9 and f2[30] > 0.9
    s3 = np.concatenate([r, q])              # n - m = 10: diagonal +10 is inside the strip
    f3 = bf.pair_features(q, s3)
    assert f3[14] > 0.9
    empty = bf.pair_features(np.zeros(0, np.uint8), q)
    assert np.all(empty[4:31] == 0) and empty[31] == 1 and empty[0] == 0


# ---------------------------------------------------------------- network
def _rand_params(rng):
    return synth.mlp_init(int(rng.integers(1 << 30))).astype(np.float64) + \
        rng.normal(0, 0.05, size=mlp.NPARAMS)


def test_param_layout():
    assert mlp.NPARAMS == synth.MLP_NPARAMS == 64 * 32 + 64 + 64 * 64 + 64 + 64 + 1
    P = mlp.unpack(np.arange(mlp.NPARAMS, dtype=np.float64))
    assert P["W1"][1, 0] == 32 and P["b1"][0] == 2048 and P["W2"][0, 1] == 2048 + 64 + 1
    assert P["b3"][0] == mlp.NPARAMS - 1


def test_forward_closed_form():
    p = np.zeros(mlp.NPARAMS)
    P = mlp.unpack(p)
    P["W1"][:32, :] = np.eye(32)
    P["W2"][:] = np.eye(64)
    P["w3"][:] = 1.0
    P["b3"][0] = 0.5
    X = np.random.default_rng(1).normal(size=(5, 32))
    y, _ = mlp.forward(p, X)
    np.testing.assert_allclose(y, np.maximum(X, 0).sum(axis=1) + 0.5, rtol=0, atol=1e-12)
    P["b2"][:] = -100.0                      # every hidden unit off: y = b3
    y, _ = mlp.forward(p, X)
    assert np.all(y == 0.5)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    p = _rand_params(rng)
    X = rng.uniform(0, 1, size=(7, 32))
    t = rng.uniform(0, 12, size=7)
    L, g = mlp.loss_grad(p, X, t)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 300, replace=False), [mlp.NPARAMS - 1]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.NPARAMS)
        e[k] = h
        num = (mlp.loss_grad(p + e, X, t)[0] - mlp.loss_grad(p - e, X, t)[0]) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)), (k, num, g[k])
    y, _ = mlp.forward(p, X)
    assert L == pytest.approx(0.5 * np.mean((y - t) ** 2), rel=1e-12)
    assert mlp.loss_grad(p, X, y)[0] == 0.0


def test_adam_closed_forms():
    rng = np.random.default_rng(3)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    z = np.zeros(50)
    w1, m1, v1 = mlp.adam_step(w, z, z, g, 1, 1e-2, eps=0.0)
    np.testing.assert_allclose(w1, w - 1e-2 * np.sign(g), rtol=0, atol=1e-15)
    w2, _, _ = mlp.adam_step(w1, m1, v1, g, 2, 1e-2, eps=0.0)   # constant gradient: same step
    np.testing.assert_allclose(w2, w - 2e-2 * np.sign(g), rtol=0, atol=1e-14)
    w3, _, _ = mlp.adam_step(w, z, z, np.zeros(50), 1, 1e-2)
    assert np.all(w3 == w)


def test_bf16_round_to_nearest_even():
    f = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.0, 0.0,
                  2 - 2 ** -9, 3.0e38, 1.0e-40], dtype=np.float32)
    bits = mlp.bf16_bits(f)
    assert list(bits[:7]) == [0x3F80, 0x3F80, 0x3F82, 0x3F81, 0xC000, 0x0000, 0x4000]
    assert bits[7] == 0x7F62 and bits[8] == 0x0001   # 0x7F61B1E6 rounds up, 0x000116C2 down
    back = mlp.bf16_to_f32(bits[:7])
    assert list(back) == [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.0, 0.0, 2.0]
