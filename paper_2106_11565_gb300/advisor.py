"""Parameter advisor from the query-time analysis of FLINNG (Sec. 4, Thm. 3
and the lemmas after it): the design the theory prescribes for given data
size, neighbour similarities and target error rates.

The paper's symbols and this library's differ: the paper's m (Bloom-filter
arrays, i.e. hash tables) is the library's L, and the paper's L (hashes
concatenated per array) is the library's K. Results are returned under the
library's names, with the paper's beside them.

Host-side arithmetic only (no kernels): it chooses parameters, it does not
run the method.
"""
from __future__ import annotations

import math


def gamma(s_k: float, s_k1: float) -> float:
    """Stability of a query (Def. of a gamma-stable query): log(s_k) /
    (log(s_k1) - log(s_k)), with s_k the similarity of the k-th nearest
    neighbour and s_k1 that of the (k+1)-th. Small means a clear gap."""
    if not (0.0 < s_k1 < s_k <= 1.0):
        raise ValueError("need 0 < s_k1 < s_k <= 1")
    return math.log(s_k) / (math.log(s_k1) - math.log(s_k))


def cells_per_repetition(n: int) -> int:
    """B = 2 sqrt(N), the choice that makes the filter error independent of N."""
    return max(1, int(round(2.0 * math.sqrt(n))))


def bits_per_table(n: int, b: int, s_k: float, s_k1: float) -> int:
    """The smallest positive integer K (the paper's L) with
    s_k^K >= 2 (N/B) s_k1^K: positives' per-table collision rate at least twice
    the negatives' expected rate in a cell of N/B points."""
    if not (0.0 < s_k1 < s_k <= 1.0):
        raise ValueError("need 0 < s_k1 < s_k <= 1")
    if s_k == 1.0 and s_k1 == 0.0:
        return 1
    # closed form of s_k^K = 2 (N/B) s_k1^K, then the first integer at or above it
    k = max(1, math.ceil(math.log(2.0 * n / b) / (math.log(s_k) - math.log(s_k1))))
    while k > 1 and s_k ** (k - 1) >= 2.0 * n / b * s_k1 ** (k - 1):
        k -= 1
    while s_k ** k < 2.0 * n / b * s_k1 ** k:
        k += 1
    return k


def design(n: int, s_k: float, s_k1: float, p_target: float, q_target: float) -> dict:
    """Thm. 3's parameters for a distance-sensitive Bloom filter per cell.

    n: points; s_k, s_k1: similarities of the k-th and (k+1)-th neighbours;
    p_target, q_target: wanted true and false positive rates of one filter.
    Returns B, K (paper's L), L (paper's m), the threshold t (collisions),
    alpha (the common bound: q <= alpha, p >= 1 - alpha) and gamma."""
    if not (0.0 < q_target < 1.0 and 0.0 < p_target < 1.0):
        raise ValueError("p_target and q_target must lie in (0, 1)")
    b = cells_per_repetition(n)
    k = bits_per_table(n, b, s_k, s_k1)
    g = gamma(s_k, s_k1)
    # m = -8 log(min(q', 1 - p')) N^gamma, in logs: unstable queries overflow it
    log_m = math.log(-8.0 * math.log(min(q_target, 1.0 - p_target))) + g * math.log(n)
    m = math.exp(log_m) if log_m < 700.0 else math.inf
    pos = s_k ** k                      # per-table collision rate of a positive cell
    neg = (n / b) * s_k1 ** k           # expected rate of a negative cell (union over N/B points)
    t = m * (neg + pos) / 2.0           # midway between the two
    alpha = math.exp(-2.0 * m * ((pos - neg) / 2.0) ** 2) if math.isfinite(m) else 0.0
    return {"B": b, "K": k, "L": int(math.ceil(m)) if math.isfinite(m) else None, "t": t, "alpha": alpha,
            "gamma": g, "log10_L": log_m / math.log(10.0),
            "paper": {"B": b, "L": k, "m": m, "t": t},
            "positive_rate": pos, "negative_rate": neg,
            "query_cost_mL": m * k}


def nearest_neighbour_design(n: int, delta: float) -> dict:
    """The cell-wise rates and repetitions that solve the randomized nearest
    neighbour problem with failure probability delta (the lemma after Thm. 3):
    R = log(1/delta) / (log(4.80 N^1/2) - log(2 e^2 + 3.44 N^1/2)),
    p = 1 - delta / (2 R), q = N^-1/2. The lemma assumes N >= 150 and
    R >= 10 log N; 'assumptions_hold' says whether they do."""
    if not (0.0 < delta < 1.0) or n < 2:
        raise ValueError("need n >= 2 and 0 < delta < 1")
    sq = math.sqrt(n)
    den = math.log(4.80 * sq) - math.log(2.0 * math.e ** 2 + 3.44 * sq)
    if den <= 0.0:
        raise ValueError("N too small for the lemma's R (the denominator is not positive)")
    r = math.log(1.0 / delta) / den
    return {"R": r, "R_int": int(math.ceil(r)), "p": 1.0 - delta / (2.0 * r), "q": 1.0 / sq,
            "assumptions_hold": n >= 150 and r >= 10.0 * math.log(n)}
