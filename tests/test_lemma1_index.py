"""Lemma 1 on FLINNG's own index (Sec. 4): the B x R grid of Alg. 1 with the
real group tests of Sec. 3.3 - a cell tests positive for query y when at
least t of the L shared LSH tables put y in a bucket holding a member of the
cell - on planted-neighbour data: |K| near neighbours of y ("positives")
among N points. Every trial draws fresh Alg. 1 permutations and fresh LSH
functions. Measured per test: p = Pr[a cell holding a positive fires],
q = Pr[a cell holding none fires]; measured per point: the report rate of
positives and of negatives (all R of its cells fire, Alg. 2's AND). The
lemma assumes i.i.d. tests; the real tests share their LSH functions, yet
the report rates must keep to its statements: positives at least p^R,
negatives at most the lemma's bound, and near the exact rate under
independence (p (1 - h0) + q h0)^R, h0 the hypergeometric probability that
a negative's group holds no positive. CPU only (the oracle)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_11565_gb300 import workloads as WL


def h0(n: int, b: int, k: int) -> float:
    return math.comb(n - n // b, k) / math.comb(n - 1, k)


def lemma_bound(n: int, b: int, k: int, p: float, q: float, r: int) -> float:
    a = n * (b - 1) / (b * (n - 1))
    return (q * (math.e * a) ** k + p * (1 - (a / math.e) ** k)) ** r


def planted_vectors(rng, n, d, k, cos):
    y = rng.standard_normal(d)
    y /= np.linalg.norm(y)
    x = rng.standard_normal((n, d))
    # positives: unit vectors at cosine `cos` to y
    z = rng.standard_normal((k, d))
    z -= (z @ y)[:, None] * y[None, :]
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    x[:k] = cos * y[None, :] + math.sqrt(1 - cos * cos) * z
    return x.astype(np.float32), y.astype(np.float32)[None, :]


def planted_sets(rng, n, size, k, share):
    universe = 1 << 30
    q = rng.choice(universe, size, replace=False).astype(np.uint32)
    rows = []
    for i in range(n):
        if i < k:
            keep = rng.choice(q, int(share * size), replace=False)
            rows.append(np.concatenate([keep, rng.integers(0, universe, size - len(keep))]).astype(np.uint32))
        else:
            rows.append(rng.integers(0, universe, size).astype(np.uint32))
    off, el = WL.csr_from_rows(rows)
    return (off, el), (np.array([0, size], np.uint64), q)


def report_rates(metric, n, k, R, B, L, K, W, t, trials, seed):
    rng = np.random.default_rng(seed)
    fires = {True: [0, 0], False: [0, 0]}           # cells with / without a positive: fired, total
    rep = {True: 0, False: 0}
    for tr in range(trials):
        if metric == "cosine":
            x, y = planted_vectors(rng, n, 64, k, 0.95)
            w = WL.srp_projections(seed * 1000 + tr, L * K, 64)
            bx = O.srp_codes(x, w, L, K)
            by = O.srp_codes(y, w, L, K)[0]
        else:
            pts, qs = planted_sets(rng, n, 200, k, 0.6)
            dp = WL.doph_params(seed * 1000 + tr, L, K)
            v = O.doph(pts[0], pts[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
            bx = O.minhash_buckets(v, L, K, dp["bucket_a"], dp["bucket_c"], W)
            vq = O.doph(qs[0], qs[1], L * K, dp["doph_a"], dp["doph_b"], dp["doph_seed"])
            by = O.minhash_buckets(vq, L, K, dp["bucket_a"], dp["bucket_c"], W)[0]
        gid = O.groups(WL.group_permutations(seed * 1000 + tr, R, n), B)
        cnt = O.counts_direct(bx, gid, B, by).astype(np.int64)           # B*R cell counts
        cells = gid.astype(np.int64) + (np.arange(R) * B)[None, :]
        has_pos = np.zeros(B * R, bool)
        has_pos[np.unique(cells[:k])] = True
        fire = cnt >= t
        for hp in (True, False):
            fires[hp][0] += int(fire[has_pos == hp].sum())
            fires[hp][1] += int((has_pos == hp).sum())
        report = fire[cells].all(axis=1)
        rep[True] += int(report[:k].sum())
        rep[False] += int(report[k:].sum())
    p = fires[True][0] / fires[True][1]
    q = fires[False][0] / fires[False][1]
    return p, q, rep[True] / (k * trials), rep[False] / ((n - k) * trials)


@pytest.mark.parametrize("k", [1, 4])
@pytest.mark.parametrize("metric,R", [("cosine", 2), ("cosine", 3), ("cosine", 4),
                                      ("jaccard", 2), ("jaccard", 3), ("jaccard", 4)])
def test_lemma1_on_the_real_index(metric, R, k):
    n, B, trials = 1200, 30, 100
    if metric == "cosine":
        L, K, W, t = 16, 10, 10, 3
    else:
        L, K, W, t = 16, 2, 12, 2
    p, q, pos, neg = report_rates(metric, n, k, R, B, L, K, W, t, trials, seed=7 + R + 10 * k)
    sd_pos = math.sqrt(max(pos * (1 - pos), 1e-4) / (k * trials))
    sd_neg = math.sqrt(max(neg * (1 - neg), 1e-6) / ((n - k) * trials))
    indep = (p * (1 - h0(n, B, k)) + q * h0(n, B, k)) ** R
    bound = lemma_bound(n, B, k, p, q, R)
    assert 0.5 < p and q < 0.2, (p, q)                  # the tests separate positives
    assert pos >= p ** R - 4 * sd_pos, (pos, p ** R)
    assert neg <= bound + 4 * sd_neg, (neg, bound)
    assert abs(neg - indep) <= 4 * sd_neg + 0.5 * indep, (neg, indep)
    if k == 1:
        assert bound < 1.0                                  # the nearest-neighbour case: not vacuous
