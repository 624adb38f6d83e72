"""The parameter advisor against the relations Thm. 3 derives its choices from
(no GPU)."""
import math

import numpy as np
import pytest

from paper_2106_11565_gb300 import advisor as A

CASES = [(10_000, 0.9, 0.8), (100_000, 0.5, 0.3), (10**7, 0.95, 0.9), (150, 0.7, 0.2), (10**6, 0.3, 0.29)]


@pytest.mark.parametrize("n,s_k,s_k1", CASES)
def test_bits_per_table_is_the_smallest_separating_integer(n, s_k, s_k1):
    b = A.cells_per_repetition(n)
    assert abs(b - 2 * math.sqrt(n)) <= 0.5
    k = A.bits_per_table(n, b, s_k, s_k1)
    assert s_k ** k >= 2 * n / b * s_k1 ** k
    assert k == 1 or s_k ** (k - 1) < 2 * n / b * s_k1 ** (k - 1)
    # with B = 2 sqrt(N) the separating exponent is (1/2) log N / (log s_k - log s_k1)
    k_star = 0.5 * math.log(n) / (math.log(s_k) - math.log(s_k1))
    assert abs(2 * n / b - math.sqrt(n)) / math.sqrt(n) < 3e-2     # B is rounded to an integer
    assert k_star - 1.05 <= k <= max(1, math.ceil(k_star) + 1)


@pytest.mark.parametrize("n,s_k,s_k1", CASES)
@pytest.mark.parametrize("p,q", [(0.99, 0.01), (0.9, 0.001)])
def test_design_relations(n, s_k, s_k1, p, q):
    d = A.design(n, s_k, s_k1, p, q)
    m, k, g = d["paper"]["m"], d["K"], d["gamma"]
    # m makes the gamma-stable bound on alpha equal to min(q', 1 - p')
    assert math.isclose(math.exp(-m * n ** (-g) / 8), min(q, 1 - p), rel_tol=1e-9)
    # t / m lies strictly between the negative and the positive collision rates
    pos, neg = d["positive_rate"], d["negative_rate"]
    assert neg * m < d["t"] < pos * m
    # alpha is the common bound; the choice of K halves the gap at worst
    assert math.isclose(d["alpha"], math.exp(-2 * m * ((pos - neg) / 2) ** 2), rel_tol=1e-12)
    assert d["alpha"] <= math.exp(-m * pos ** 2 / 8) * (1 + 1e-12)
    assert d["L"] == math.ceil(m) and d["query_cost_mL"] == pytest.approx(m * k)


@pytest.mark.parametrize("n,s_k,s_k1", CASES)
def test_gamma_and_the_continuous_exponent(n, s_k, s_k1):
    g = A.gamma(s_k, s_k1)
    assert g > 0
    # at the continuous exponent the positive rate is exactly N^(-gamma/2)
    k_star = 0.5 * math.log(n) / (math.log(s_k) - math.log(s_k1))
    assert math.isclose(s_k ** k_star, n ** (-g / 2), rel_tol=1e-9)


def test_gamma_rejects_unordered_similarities():
    with pytest.raises(ValueError):
        A.gamma(0.5, 0.5)
    with pytest.raises(ValueError):
        A.gamma(0.4, 0.6)


@pytest.mark.parametrize("n,delta", [(150, 1e-3), (10**4, 1e-6), (10**8, 0.01), (10**6, 1e-30)])
def test_nearest_neighbour_design(n, delta):
    d = A.nearest_neighbour_design(n, delta)
    r = d["R"]
    assert math.isclose(r, math.log(1 / delta) /
                        (math.log(4.80 * math.sqrt(n)) - math.log(2 * math.e ** 2 + 3.44 * math.sqrt(n))))
    # p = 1 - delta / 2R keeps the miss probability 1 - p^R within delta / 2 (Bernoulli)
    assert 1 - d["p"] ** r <= delta / 2 + 1e-15
    assert d["q"] == pytest.approx(n ** -0.5)
    assert d["assumptions_hold"] == (n >= 150 and r >= 10 * math.log(n))


def test_design_on_a_measured_neighbour_gap():
    """Inputs a user would take from data: the k-th and (k+1)-th exact
    similarities of sampled queries (here a synthetic gap)."""
    rng = np.random.default_rng(3)
    sims = np.sort(rng.uniform(0.2, 0.9, size=(50, 11)), axis=1)[:, ::-1]
    s_k, s_k1 = float(np.median(sims[:, 9])), float(np.median(sims[:, 10]))
    d = A.design(100_000, s_k, s_k1, 0.99, 0.01)
    assert d["K"] >= 1 and d["L"] >= 1 and 0 < d["alpha"] < 1


def test_unstable_query_asks_for_unbounded_tables():
    """A near-tie between the k-th and (k+1)-th neighbours (large gamma): the
    table count overflows and is reported as unbounded, not as a number."""
    d = A.design(10_000, 0.99067, 0.99061, 0.99, 0.01)
    assert d["gamma"] > 100 and d["L"] is None and d["log10_L"] > 300
