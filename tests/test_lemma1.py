"""Lemma 1 statistical harness: the B x R grid of Alg. 1 with i.i.d. tests
(true positive rate p, false positive rate q) and the AND over R of Alg. 2.
Measured report rates are compared with p^R for positives and, for
negatives, with the exact per-repetition rate p (1 - h0) + q h0 (h0: the
hypergeometric probability that a negative's group holds no positive) and
with the lemma's upper bound. No GPU: the groups are Alg. 1's (oracle)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_11565_gb300 import workloads as WL


def h0(n: int, b: int, k: int) -> float:
    """Pr[a negative's group holds no positive] = C(N - N/B, |K|) / C(N - 1, |K|)."""
    return math.comb(n - n // b, k) / math.comb(n - 1, k)


def lemma_bound(n: int, b: int, k: int, p: float, q: float, r: int) -> float:
    a = n * (b - 1) / (b * (n - 1))
    return (q * (math.e * a) ** k + p * (1 - (a / math.e) ** k)) ** r


@pytest.mark.parametrize("n,b,r,k,p,q", [(2000, 40, 3, 5, 0.9, 0.05), (1200, 60, 2, 1, 0.8, 0.2),
                                          (3000, 30, 4, 12, 0.95, 0.1)])
def test_report_rates_match_lemma1(n, b, r, k, p, q):
    trials = 400
    rng = np.random.default_rng([n, b, r, k])
    pos = np.zeros(n, bool)
    pos[rng.choice(n, k, replace=False)] = True
    rep_pos = rep_neg = 0
    for tr in range(trials):
        gid = O.groups(WL.group_permutations(1000 + tr, r, n), b).astype(np.int64)   # n x r
        cells = gid + (np.arange(r) * b)[None, :]
        has_pos = np.zeros(b * r, bool)
        has_pos[np.unique(cells[pos])] = True
        test = np.where(has_pos, rng.random(b * r) < p, rng.random(b * r) < q)
        report = test[cells].all(axis=1)                       # AND over the R repetitions
        rep_pos += int(report[pos].sum())
        rep_neg += int(report[~pos].sum())
    n_pos, n_neg = trials * k, trials * (n - k)
    tpr, fpr = rep_pos / n_pos, rep_neg / n_neg
    # positives: every group holding x holds a positive, so exactly p^R
    sd = math.sqrt(p ** r * (1 - p ** r) / n_pos)
    assert abs(tpr - p ** r) <= 4 * sd + 1e-12
    # negatives: exact hypergeometric rate per repetition, repetitions independent
    z = h0(n, b, k)
    exact = (p * (1 - z) + q * z) ** r
    # reports of negatives within one trial are correlated (shared groups): a
    # loose 6 sigma on the per-trial binomial count
    sd_n = math.sqrt(exact * (1 - exact) / n_neg) * math.sqrt(n / b)
    assert abs(fpr - exact) <= 6 * sd_n + 1e-12
    assert exact <= lemma_bound(n, b, k, p, q, r) * (1 + 1e-12)


def test_hypergeometric_zero_by_brute_force():
    """h0 against direct enumeration on a tiny case: all placements of a
    negative's N/B - 1 cell-mates among the other N - 1 points."""
    from itertools import combinations
    n, b, k = 12, 3, 2
    size = n // b
    others = list(range(1, n))              # point 0 is the negative; positives are points 1..k
    good = total = 0
    for mates in combinations(others, size - 1):
        total += 1
        good += all(m > k for m in mates)
    assert math.isclose(h0(n, b, k), good / total)
