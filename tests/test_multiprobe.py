"""Multi-probe counts in the oracle: in table l the query probes its bucket
and the P - 1 buckets with one of code bits 0 .. P-2 flipped; a cell counts
table l once if any member's bucket is a probe. Pinned by a hand-worked case,
by P = 1 reducing to the single-probe definition, by a set-based brute force
written apart from the oracle, and by monotonicity in P with counts <= L."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_11565_gb300 import workloads as WL


def test_hand_case():
    # three points in their own cells (R = 1, B = 3), two tables of 2-bit codes
    gid = O.groups(np.array([[0, 1, 2]], np.uint32), 3)
    assert gid[:, 0].tolist() == [0, 1, 2]
    buckets = np.array([[0b01, 0b11], [0b10, 0b01], [0b11, 0b00]], np.uint32)
    q = np.array([0b00, 0b11], np.uint32)
    # P = 1: the query's own buckets 00 and 11: x0 shares table 1's
    assert O.counts_multiprobe(buckets, gid, 3, q, 1).tolist() == [1, 0, 0]
    # P = 2: probes {00, 01} in table 0 and {11, 10} in table 1: only x0 (01, 11)
    assert O.counts_multiprobe(buckets, gid, 3, q, 2).tolist() == [2, 0, 0]
    # P = 3 adds bit 1: {00, 01, 10} and {11, 10, 01}: x0 and x1 in both tables
    assert O.counts_multiprobe(buckets, gid, 3, q, 3).tolist() == [2, 2, 0]


def brute(buckets, gid, B, q, P):
    N, L = buckets.shape
    R = gid.shape[1]
    cnt = np.zeros(B * R, np.int64)
    for l in range(L):
        probes = {int(q[l])} | {int(q[l]) ^ (1 << j) for j in range(P - 1)}
        cells = set()
        for x in range(N):
            if int(buckets[x, l]) in probes:
                cells |= {r * B + int(gid[x, r]) for r in range(R)}
        for c in cells:
            cnt[c] += 1
    return cnt


@pytest.mark.parametrize("seed", range(12))
def test_multiprobe_counts(seed):
    rng = np.random.default_rng(1500 + seed)
    N, R, B, L, K = int(rng.integers(1, 80)), int(rng.integers(1, 4)), int(rng.integers(1, 12)), \
        int(rng.integers(1, 9)), int(rng.integers(1, 7))
    buckets = rng.integers(0, 1 << K, size=(N, L)).astype(np.uint32)
    q = rng.integers(0, 1 << K, size=L).astype(np.uint32)
    gid = O.groups(WL.group_permutations(seed, R, N), B)
    assert np.array_equal(O.counts_multiprobe(buckets, gid, B, q, 1), O.counts_direct(buckets, gid, B, q))
    prev = None
    for P in range(1, K + 2):
        c = O.counts_multiprobe(buckets, gid, B, q, P)
        assert np.array_equal(c, brute(buckets, gid, B, q, P))
        assert c.max(initial=0) <= L
        if prev is not None:
            assert np.all(c >= prev)
        prev = c
