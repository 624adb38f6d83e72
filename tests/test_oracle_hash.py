"""Pins for the oracle's hashing steps (CPU only).

Each check compares the oracle with something other than itself: published
generator outputs, exact rational arithmetic, hand-derived cases, invariants,
and the closed-form collision probabilities of the two LSH families
(Sec. 3.2: s(x, y) = sim(x, y); concatenation gives s^K).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ splitmix64

def test_splitmix64_published_sequence():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_1234567.txt"))
            if l.strip() and not l.startswith("#")]
    g = 0x9E3779B97F4A7C15
    for i, v in enumerate(vals):
        # the reference generator adds the increment to its state, then mixes
        state = (1234567 + i * g) % (1 << 64)
        assert O.splitmix64(state) == v


# ------------------------------------------------------------ exact sign

def _exact_sign(a, b):
    s = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in
            zip(np.asarray(a, np.float32), np.asarray(b, np.float32)))
    return (s > 0) - (s < 0)


@pytest.mark.parametrize("vec,expect", [
    ([2.0 ** 60, 1.0, -2.0 ** 60], 1),     # fp64 in order gives 0; exact is +1
    ([2.0 ** 60, -1.0, -2.0 ** 60], -1),
    ([2.0 ** 60, -2.0 ** 60, 0.0], 0),
    ([0.0, 0.0, 0.0], 0),
    ([2.0 ** -149, 0.0, 0.0], 1),          # product 2^-298, smallest possible
    ([-(2.0 ** -149), 0.0, 0.0], -1),
    ([3.0e38, 3.0e38, -3.0e38], 1),        # products near 2^256
])
def test_exact_dot_sign_hand_cases(vec, expect):
    a = np.array(vec, np.float32)
    b = np.ones_like(a)
    if vec[0] in (2.0 ** -149, -(2.0 ** -149)):
        b = np.array([2.0 ** -149, 1.0, 1.0], np.float32)
    if vec[0] == 3.0e38:
        b = np.array([3.0e38, 3.0e38, 3.0e38], np.float32)
    assert O.exact_dot_sign(a, b) == expect == _exact_sign(a, b)


def test_exact_dot_sign_matches_rationals_on_cancellation():
    rng = np.random.default_rng(5)
    for trial in range(300):
        d = int(rng.integers(1, 40))
        a = (rng.standard_normal(d) * 2.0 ** rng.integers(-30, 30, size=d)).astype(np.float32)
        b = (rng.standard_normal(d) * 2.0 ** rng.integers(-30, 30, size=d)).astype(np.float32)
        if trial % 2 == 0 and d >= 2:   # force near-total cancellation
            a[-1] = np.float32(-float(np.dot(a[:-1].astype(np.float64), b[:-1])) / float(b[-1]))
        assert np.all(np.isfinite(a))
        assert O.exact_dot_sign(a, b) == _exact_sign(a, b)


# ------------------------------------------------------------ SRP

def test_srp_bit_layout_by_hand():
    # rows 0..3 pick coordinates, rows 4..7 pick negated coordinates
    x = np.array([[1.0, -2.0, 3.0, -4.0], [0.0, 0.0, 0.0, 0.0]], np.float32)
    w = np.concatenate([np.eye(4), -np.eye(4)]).astype(np.float32)
    codes = O.srp_codes(x, w, L=2, K=4)
    # point 0: projections 1,-2,3,-4 -> bits 1,0,1,0 -> 0b0101; negated 0b1010
    assert codes[0].tolist() == [0b0101, 0b1010]
    # zero projection: bit = (p > 0) = 0
    assert codes[1].tolist() == [0, 0]


def test_srp_codes_equal_exact_signs():
    rng = np.random.default_rng(7)
    n, d, L, K = 40, 24, 3, 5
    x = rng.standard_normal((n, d)).astype(np.float32)
    w = rng.standard_normal((L * K, d)).astype(np.float32)
    # plant projections that cancel exactly or nearly exactly
    for i in range(0, n, 4):
        j = i % (L * K)
        x[i, -1] = np.float32(-float(np.dot(w[j, :-1].astype(np.float64), x[i, :-1])) / float(w[j, -1]))
    codes, proj, n_exact = O.srp_codes(x, w, L, K, want_proj=True)
    for i in range(n):
        for j in range(L * K):
            bit = (int(codes[i, j // K]) >> (j % K)) & 1
            assert bit == (_exact_sign(w[j], x[i]) > 0)
    # fp64 projections agree with a float64 library dot to rounding
    ref = x.astype(np.float64) @ w.astype(np.float64).T
    scale = np.abs(x).astype(np.float64) @ np.abs(w).astype(np.float64).T
    assert np.all(np.abs(proj - ref) <= 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("theta", [0.2, 0.7, 1.3, 2.1, 2.9])
def test_srp_collision_rate_is_one_minus_theta_over_pi(theta):
    rng = np.random.default_rng(int(theta * 1000))
    d = 32
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    v = rng.standard_normal(d)
    v -= v.dot(u) * u
    v /= np.linalg.norm(v)
    x = np.stack([u, math.cos(theta) * u + math.sin(theta) * v]).astype(np.float32)
    L, K = 512, 16
    wmat = rng.standard_normal((L * K, d)).astype(np.float32)
    codes = O.srp_codes(x, wmat, L, K)
    eq = ~(codes[0] ^ codes[1])
    bits = np.unpackbits(eq.view(np.uint8).reshape(L, 4), axis=1, bitorder="little")[:, :K]
    frac = bits.mean()
    p = 1.0 - theta / math.pi
    sigma = math.sqrt(p * (1 - p) / (L * K))
    assert abs(frac - p) < 4 * sigma + 1e-3
    # concatenation trick: a table collides when all K bits agree, prob p^K
    tab = (codes[0] == codes[1]).mean()
    pk = p ** K
    assert abs(tab - pk) < 4 * math.sqrt(pk * (1 - pk) / L) + 2e-3


# ------------------------------------------------------------ DOPH

def _sets(rows):
    off = np.zeros(len(rows) + 1, np.uint64)
    off[1:] = np.cumsum([len(r) for r in rows])
    el = np.concatenate([np.asarray(r, np.uint32) for r in rows]) if rows else np.zeros(0, np.uint32)
    return off, el


def test_doph_hand_case():
    # a = 1, b = 0: pi(e) = e; nb = 4 bins are the top two bits of pi(e)
    A = [0x10000000, 0x50000000, 0x60000000]
    off, el = _sets([A])
    seed = 99
    v = O.doph(off, el, 4, 1, 0, seed)[0]
    assert v[0] == 0x10000000                 # bin 0 holds 0x1...
    assert v[1] == 0x50000000                 # bin 1 holds 0x5... and 0x6...; min
    # bins 2 and 3 are empty: each copies the first non-empty bin that the
    # splitmix64 sequence seed ^ (i << 32 | attempt), attempt = 1, 2, ... hits
    for i in (2, 3):
        for att in range(1, 100):
            j = O.splitmix64(seed ^ ((i << 32) | att)) % 4
            if j in (0, 1):
                break
        assert v[i] == v[j]


def test_doph_invariants():
    rng = np.random.default_rng(3)
    A = rng.choice(1 << 32, size=300, replace=False).astype(np.uint32)
    B = rng.choice(1 << 32, size=300, replace=False).astype(np.uint32)
    B = np.setdiff1d(B, A)
    rows = [A, A[::-1].copy(), np.concatenate([A, A[:50]]), B, np.zeros(0, np.uint32), A[:1]]
    off, el = _sets(rows)
    a, b, s = 0x9E3779B1, 12345, 777
    v = O.doph(off, el, 64, a, b, s)
    assert np.array_equal(v[0], v[1])          # order does not matter
    assert np.array_equal(v[0], v[2])          # duplicates do not matter
    assert not np.any(v[0] == v[3])            # disjoint sets never collide
    assert np.all(v[4] == 0xFFFFFFFF)          # empty set
    e = (a * int(A[0]) + b) % (1 << 32)        # one element: every bin holds pi(e)
    assert np.all(v[5] == e)
    # every value is pi of some element of its set
    pis = set(((a * A.astype(np.uint64) + b) % (1 << 32)).tolist())
    assert set(v[0].tolist()) <= pis


@pytest.mark.parametrize("size,inter", [(200, 100), (200, 40), (12, 6)])
def test_doph_collision_rate_is_jaccard(size, inter):
    rng = np.random.default_rng(size * 1000 + inter)
    pool = rng.choice(1 << 32, size=2 * size, replace=False).astype(np.uint32)
    A = pool[:size]
    B = np.concatenate([pool[:inter], pool[size:2 * size - inter]])
    J = inter / (2 * size - inter)
    off, el = _sets([A, B])
    draws = 1500
    means = np.empty(draws)
    for t in range(draws):
        a = int(rng.integers(0, 1 << 32)) | 1
        b = int(rng.integers(0, 1 << 32))
        s = int(rng.integers(0, 1 << 62))
        v = O.doph(off, el, 64, a, b, s)
        means[t] = np.mean(v[0] == v[1])
    m = means.mean()
    se = means.std(ddof=1) / math.sqrt(draws)
    assert abs(m - J) < 4 * se + 0.01, (m, J, se)


# ------------------------------------------------------------ buckets

def test_minhash_bucket_hand_case():
    # multiplier 2^32 + 1 and offset 0 put v itself in the top 32 bits, so the
    # W-bit bucket is the top W bits of v
    v = np.array([[0xDEADBEEF], [0x00000001], [0xFFFFFFFF]], np.uint32)
    ba = np.array([[(1 << 32) | 1]], np.uint64)
    bc = np.array([0], np.uint64)
    for W in (1, 8, 17, 32):
        out = O.minhash_buckets(v, 1, 1, ba, bc, W)
        assert out[:, 0].tolist() == [int(x) >> (32 - W) for x in v[:, 0]]


def test_minhash_bucket_range_and_determinism():
    rng = np.random.default_rng(11)
    L, K, W = 8, 3, 17
    v = rng.integers(0, 1 << 32, size=(500, L * K), dtype=np.uint64).astype(np.uint32)
    v[1] = v[0]
    ba = rng.integers(0, 1 << 63, size=(L, K), dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    bc = rng.integers(0, 1 << 63, size=(L,), dtype=np.uint64)
    out = O.minhash_buckets(v, L, K, ba, bc, W)
    assert out.max() < (1 << W)
    assert np.array_equal(out[0], out[1])
    # buckets spread over the range: no value holds more than 1% of 4000 draws
    assert np.bincount(out.ravel()).max() < 40
